"""Seeded synthetic inputs: reaction networks, parameter sets and BLTL properties.

This module is shared by the tests, the benchmark and the CPU oracle.  It only
*describes* inputs (species, reactions, rate constants, initial counts, atoms
and formula trees); it performs none of the method's arithmetic (no
propensities, no simulation, no monitoring, no interval computation).

Conventions (all arrays are numpy):

* ``reactants``  int32 [R, 2]  species index of each reactant slot or -1.
  Two equal ids mean a homodimer reaction S_i + S_i -> ...
* ``stoich``     int32 [R, S]  net change v_ji of species i when R_j fires.
* ``rates``      float64 [n_inst, R]  stochastic rate constants c_j.
* ``x0``         int32 [n_inst, S]  initial molecule counts.

A property is ``Property(atoms, formula)`` where each atom is a linear
constraint ``sum_i coef[i] * x_i  <op>  bound`` with integer coefficients and
``formula`` is a tree of tuples:

  ('true',) ('false',) ('atom', k) ('not', f) ('and', f, g) ('or', f, g)
  ('implies', f, g) ('U', a, b, f, g) ('F', a, b, f) ('G', a, b, f) ('X', a, b, f)

which is the BLTLc grammar of Sec. 3.1 restricted to linear atoms over counts,
with closed time intervals [a, b].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

OPS = ('<', '<=', '>=', '>', '==', '!=')


TOKENS = ('x', 'c', '+', '-', '*', '/', 'sqrt', 'pow')


@dataclasses.dataclass
class Atom:
    """``sum_i coef[i] x_i <op> bound``, or, when ``lhs`` is given, the
    arithmetic atom ``lhs <op> rhs`` (Sec. 3.1's val <| val): each side a
    postfix program of tokens ('x', species index), ('c', constant), ('+',),
    ('-',), ('*',), ('/',), ('sqrt',), ('pow', n)."""
    coef: np.ndarray  # int32 [S]
    op: str
    bound: float
    lhs: list = None
    rhs: list = None

    def __post_init__(self):
        self.coef = np.ascontiguousarray(self.coef, dtype=np.int32)
        if self.op not in OPS:
            raise ValueError(f"unknown comparison {self.op!r}")
        self.bound = float(self.bound)
        for side in (self.lhs, self.rhs):
            for t in side or []:
                if t[0] not in TOKENS:
                    raise ValueError(f"unknown token {t!r}")


@dataclasses.dataclass
class Property:
    atoms: List[Atom]
    formula: tuple
    text: str = ""


@dataclasses.dataclass
class Model:
    """One reaction network with ``n_inst`` parameter sets (rates, x0)."""
    name: str
    species: List[str]
    reactants: np.ndarray
    stoich: np.ndarray
    rates: np.ndarray
    x0: np.ndarray
    # rate-law factors beyond mass action, shared by all instances: tuples
    # (reaction k, species m, power n, a0, a1, b0, b1) multiplying a_k by
    # (a0 + a1 x_m^n) / (b0 + b1 x_m^n), applied in the listed order
    factors: list = dataclasses.field(default_factory=list)

    def __post_init__(self):
        self.reactants = np.ascontiguousarray(self.reactants, dtype=np.int32).reshape(-1, 2)
        R = self.reactants.shape[0]
        S = len(self.species)
        self.stoich = np.ascontiguousarray(self.stoich, dtype=np.int32).reshape(R, S)
        self.rates = np.ascontiguousarray(self.rates, dtype=np.float64).reshape(-1, R)
        self.x0 = np.ascontiguousarray(self.x0, dtype=np.int32).reshape(-1, S)
        if self.rates.shape[0] != self.x0.shape[0]:
            if self.x0.shape[0] == 1:
                self.x0 = np.ascontiguousarray(np.repeat(self.x0, self.rates.shape[0], axis=0))
            elif self.rates.shape[0] == 1:
                self.rates = np.ascontiguousarray(np.repeat(self.rates, self.x0.shape[0], axis=0))
            else:
                raise ValueError("rates and x0 disagree on the instance count")

    @property
    def n_species(self) -> int:
        return len(self.species)

    @property
    def n_reactions(self) -> int:
        return self.reactants.shape[0]

    @property
    def n_inst(self) -> int:
        return self.rates.shape[0]

    def instance(self, m: int) -> "Model":
        return Model(self.name, list(self.species), self.reactants, self.stoich,
                     self.rates[m:m + 1], self.x0[m:m + 1], list(self.factors))


@dataclasses.dataclass
class Batch:
    """Heterogeneous networks (one instance each) with one shared formula
    shape whose atoms may differ per instance."""
    models: List[Model]
    properties: List[Property]

    @property
    def n_inst(self) -> int:
        return len(self.models)


# ---------------------------------------------------------------------------
# helpers

def _net(species: Sequence[str], reactions: Sequence[Tuple[Sequence[str], Sequence[str]]]):
    idx = {s: i for i, s in enumerate(species)}
    R = len(reactions)
    reac = -np.ones((R, 2), np.int32)
    st = np.zeros((R, len(species)), np.int32)
    for j, (lhs, rhs) in enumerate(reactions):
        if len(lhs) > 2:
            raise ValueError("order > 2")
        for s_slot, s in enumerate(lhs):
            reac[j, s_slot] = idx[s]
            st[j, idx[s]] -= 1
        for s in rhs:
            st[j, idx[s]] += 1
    return reac, st


def expr_atom(species: Sequence[str], lhs, op: str, rhs) -> Atom:
    """Arithmetic atom ``lhs <op> rhs``; tokens ('x', name) name species."""
    idx = {s: i for i, s in enumerate(species)}

    def res(side):
        return [('x', idx[t[1]]) if t[0] == 'x' else tuple(t) for t in side]
    return Atom(np.zeros(len(species), np.int32), op, 0.0, res(lhs), res(rhs))


def atom(species: Sequence[str], terms, op: str, bound: float) -> Atom:
    """``terms`` is a species name or a dict name -> integer coefficient."""
    if isinstance(terms, str):
        terms = {terms: 1}
    coef = np.zeros(len(species), np.int32)
    for name, c in terms.items():
        coef[list(species).index(name)] = int(c)
    return Atom(coef, op, bound)


# ---------------------------------------------------------------------------
# the five workloads and the closed-form test models

def immigration_death(n_inst: int = 1) -> Tuple[Model, Property]:
    """0 -> A (c=10), A -> 0 (c=0.1), A0=0; property F[0,100](A >= 130)."""
    sp = ['A']
    reac, st = _net(sp, [([], ['A']), (['A'], [])])
    m = Model('immigration_death', sp, reac, st,
              np.tile([10.0, 0.1], (n_inst, 1)), np.zeros((n_inst, 1)))
    p = Property([atom(sp, 'A', '>=', 130)], ('F', 0.0, 100.0, ('atom', 0)), 'F[0,100](A>=130)')
    return m, p


def lotka_volterra(n_inst: int = 1) -> Tuple[Model, Property]:
    """X -> 2X (1.0), X+Y -> 2Y (0.005), Y -> 0 (0.6), X0=Y0=1000;
    property G[0,30](X>0 & Y>0)."""
    sp = ['X', 'Y']
    reac, st = _net(sp, [(['X'], ['X', 'X']), (['X', 'Y'], ['Y', 'Y']), (['Y'], [])])
    m = Model('lotka_volterra', sp, reac, st,
              np.tile([1.0, 0.005, 0.6], (n_inst, 1)), np.tile([1000, 1000], (n_inst, 1)))
    p = Property([atom(sp, 'X', '>', 0), atom(sp, 'Y', '>', 0)],
                 ('G', 0.0, 30.0, ('and', ('atom', 0), ('atom', 1))), 'G[0,30](X>0 & Y>0)')
    return m, p


def lotka_volterra_family(n_inst: int, seed: int = 1, jitter: float = 0.3) -> Tuple[Model, Property]:
    """Lotka-Volterra with every rate multiplied by a log-uniform factor in
    [1-jitter, 1+jitter] per instance (the surrogate workload)."""
    m, p = lotka_volterra(n_inst)
    rng = np.random.default_rng(seed)
    f = np.exp(rng.uniform(math.log(1 - jitter), math.log(1 + jitter), size=m.rates.shape))
    m.rates = np.ascontiguousarray(m.rates * f)
    m.name = 'lotka_volterra_family'
    return m, p


def pure_decay(A0: int = 1000, k: float = 1.0, T: float = 1.0) -> Tuple[Model, Property]:
    """A -> 0 at rate k*A.  A(T) ~ Binomial(A0, exp(-k T)).  The property
    G[0,T](A >= 0) is always true and forces simulation up to T."""
    sp = ['A']
    reac, st = _net(sp, [(['A'], [])])
    m = Model('pure_decay', sp, reac, st, [[k]], [[A0]])
    p = Property([atom(sp, 'A', '>=', 0)], ('G', 0.0, T, ('atom', 0)), f'G[0,{T}](A>=0)')
    return m, p


def immigration_only(k: float = 5.0, T: float = 10.0) -> Tuple[Model, Property]:
    """0 -> A at rate k.  The number of events in [0,T] is Poisson(k T)."""
    sp = ['A']
    reac, st = _net(sp, [([], ['A'])])
    m = Model('immigration_only', sp, reac, st, [[k]], [[0]])
    p = Property([atom(sp, 'A', '>=', 0)], ('G', 0.0, T, ('atom', 0)), f'G[0,{T}](A>=0)')
    return m, p


def dimerisation(n_inst: int = 1) -> Tuple[Model, Property]:
    """A homodimer test network: 2A -> B (c=0.002), B -> 2A (c=0.1),
    0 -> A (c=5), A0=100, B0=0; property F[0,20](B >= 40)."""
    sp = ['A', 'B']
    reac, st = _net(sp, [(['A', 'A'], ['B']), (['B'], ['A', 'A']), ([], ['A'])])
    m = Model('dimerisation', sp, reac, st, np.tile([0.002, 0.1, 5.0], (n_inst, 1)),
              np.tile([100, 0], (n_inst, 1)))
    p = Property([atom(sp, 'B', '>=', 40)], ('F', 0.0, 20.0, ('atom', 0)), 'F[0,20](B>=40)')
    return m, p


def birth_death_survival(n_inst: int = 1, b: float = 1.0, d: float = 0.8, A0: int = 5,
                         T: float = 20.0) -> Tuple[Model, Property]:
    """Linear birth-death process A -> 2A (c=b), A -> 0 (c=d) from A0;
    property G[0,T](A > 0) (the lineage survives to T).  Survivors grow like
    e^{(b-d)t}, so most of a surviving trajectory's events come late, while
    its fate is largely settled early: the setting in which a checkpoint
    predictor pays as a control variate."""
    sp = ['A']
    reac, st = _net(sp, [(['A'], ['A', 'A']), (['A'], [])])
    m = Model('birth_death_survival', sp, reac, st, np.tile([b, d], (n_inst, 1)),
              np.full((n_inst, 1), A0))
    p = Property([atom(sp, 'A', '>', 0)], ('G', 0.0, T, ('atom', 0)), f'G[0,{T}](A>0)')
    return m, p


def mm_degradation(A0: int = 40, vmax: float = 4.0, K: float = 10.0, T: float = 12.0,
                   theta: int = 8) -> Tuple[Model, Property]:
    """Michaelis-Menten degradation A -> 0 with propensity vmax A / (K + A)
    (a zeroth-order mass-action part times the factor A / (K + A));
    property F[0,T](A <= theta)."""
    sp = ['A']
    m = Model('mm_degradation', sp, [[-1, -1]], [[-1]], [[vmax]], [[A0]],
              [(0, 0, 1, 0.0, 1.0, float(K), 1.0)])
    p = Property([atom(sp, 'A', '<=', theta)], ('F', 0.0, T, ('atom', 0)), f'F[0,{T}](A<={theta})')
    return m, p


def autorepressor(n_inst: int = 1, k: float = 20.0, K: float = 30.0, n: int = 2, d: float = 0.2,
                  T: float = 40.0, theta: int = 48) -> Tuple[Model, Property]:
    """A gene repressing its own production: 0 -> A with propensity
    k K^n / (K^n + A^n) (Hill repression), A -> 0 (d A); A0 = 0; property
    F[0,T](A >= theta)."""
    sp = ['A']
    reac, st = _net(sp, [([], ['A']), (['A'], [])])
    Kn = float(K) ** n
    m = Model('autorepressor', sp, reac, st, np.tile([k, d], (n_inst, 1)), np.zeros((n_inst, 1)),
              [(0, 0, n, Kn, 0.0, Kn, 1.0)])
    p = Property([atom(sp, 'A', '>=', theta)], ('F', 0.0, T, ('atom', 0)), f'F[0,{T}](A>={theta})')
    return m, p


def factor_chain(n: int = 10, T: float = 25.0, theta: int = 10) -> Tuple[Model, Property]:
    """A conversion chain A_0 -> A_1 -> ... -> A_{n-1} (c = 1, mass action
    in A_j) whose step j is activated by A_{j+2 mod n}, factor
    (0.5 + x) / (5 + x), fed by 0 -> A_0 (c = 3) under Hill repression by
    A_{n-1}, factor 100 / (100 + x^2); A_0 = 30, property
    F[0,T](A_{n-1} >= theta).  More than 8 species: the generic kernel with
    dependency-graph updates, where a factor's species enlarges dep(j)."""
    sp = [f'A{i}' for i in range(n)]
    reactions = [([sp[j]], [sp[j + 1]]) for j in range(n - 1)] + [([], [sp[0]])]
    reac, st = _net(sp, reactions)
    rates = [1.0] * (n - 1) + [3.0]
    x0 = [30] + [0] * (n - 1)
    factors = [(j, (j + 2) % n, 1, 0.5, 1.0, 5.0, 1.0) for j in range(n - 1)]
    factors.append((n - 1, n - 1, 2, 100.0, 0.0, 100.0, 1.0))
    m = Model('factor_chain', sp, reac, st, [rates], [x0], factors)
    p = Property([atom(sp, sp[-1], '>=', theta)], ('F', 0.0, T, ('atom', 0)), f'F[0,{T}]({sp[-1]}>={theta})')
    return m, p


def sqrt_race(T: float = 15.0) -> Tuple[Model, Property]:
    """The paper's example formula (Sec. 3.1), (X1 < sqrt(X2)) U[0,T]
    (X2 >= 10 + X3), on a small network: X1 and X2 produced and degraded,
    X2 converted into X3.  0 -> X1 (1.0), X1 -> 0 (0.2 X1), 0 -> X2 (4.0),
    X2 -> X3 (0.1 X2), X3 -> 0 (0.2 X3); X1 = 2, X2 = 9, X3 = 0."""
    sp = ['X1', 'X2', 'X3']
    reac, st = _net(sp, [([], ['X1']), (['X1'], []), ([], ['X2']), (['X2'], ['X3']), (['X3'], [])])
    m = Model('sqrt_race', sp, reac, st, [[1.0, 0.2, 4.0, 0.1, 0.2]], [[2, 9, 0]])
    left = expr_atom(sp, [('x', 'X1')], '<', [('x', 'X2'), ('sqrt',)])
    right = expr_atom(sp, [('x', 'X2')], '>=', [('c', 10.0), ('x', 'X3'), ('+',)])
    p = Property([left, right], ('U', 0.0, T, ('atom', 0), ('atom', 1)),
                 f'(X1 < sqrt(X2)) U[0,{T}] (X2 >= 10 + X3)')
    return m, p


def random_networks(n_inst: int = 4096, seed: int = 3, s_range: Tuple[int, int] = (2, 32),
                    r_range: Tuple[int, int] = (4, 64), theta_above_start: bool = False) -> Batch:
    """Batched random mass-action networks.

    Per instance: S ~ U{2..32}, R ~ U{4..64} (by default; s_range and
    r_range give other bounds, inclusive); each reaction has reactant
    order uniform in {0,1,2} (species uniform, a repeated species is a
    homodimer) and 0-2 product molecules, but never more product molecules
    than reactant molecules for order >= 1 (so only zeroth-order reactions
    create mass and counts stay bounded by x0 plus the influx); rate
    constants log-uniform in [1e-3, 1]; x0 ~ U{0..200}.  Property
    F[0,50](X_k >= theta) with k uniform over species and
    theta = max(1, ceil(1.5 * mean(x0))), or, with theta_above_start,
    theta = x0_k + max(1, ceil(0.5 * mean(x0))) (never satisfied at t = 0).
    """
    rng = np.random.default_rng(seed)
    models, props = [], []
    for m in range(n_inst):
        S = int(rng.integers(s_range[0], s_range[1] + 1))
        R = int(rng.integers(r_range[0], r_range[1] + 1))
        sp = [f's{i}' for i in range(S)]
        reac = -np.ones((R, 2), np.int32)
        st = np.zeros((R, S), np.int32)
        for j in range(R):
            order = int(rng.integers(0, 3))
            for o in range(order):
                s = int(rng.integers(0, S))
                reac[j, o] = s
                st[j, s] -= 1
            n_prod = int(rng.integers(0, 3)) if order == 0 else int(rng.integers(0, order + 1))
            for _ in range(n_prod):
                st[j, int(rng.integers(0, S))] += 1
        rates = np.exp(rng.uniform(math.log(1e-3), math.log(1.0), size=R))
        x0 = rng.integers(0, 201, size=S).astype(np.int32)
        k = int(rng.integers(0, S))
        if theta_above_start:
            theta = int(x0[k]) + max(1, int(math.ceil(0.5 * float(x0.mean()))))
        else:
            theta = max(1, int(math.ceil(1.5 * float(x0.mean()))))
        models.append(Model(f'random{m}', sp, reac, st, rates[None, :], x0[None, :]))
        props.append(Property([atom(sp, sp[k], '>=', theta)], ('F', 0.0, 50.0, ('atom', 0)),
                              f'F[0,50]({sp[k]}>={theta})'))
    return Batch(models, props)


def random_networks_large(n_inst: int = 256, seed: int = 8) -> Batch:
    """Random mass-action networks with many reactions, for the selection
    step of large networks: S ~ U{16..64}, R ~ U{65..255}, otherwise the
    recipe of random_networks, with the threshold above the species'
    starting count."""
    return random_networks(n_inst, seed, s_range=(16, 64), r_range=(65, 255), theta_above_start=True)


MAPK_SPECIES = [
    'KKK', 'KKKs', 'E1', 'E2', 'KK', 'KKP', 'KKPP', 'KKPase', 'K', 'KP', 'KPP', 'KPase',
    'KKK_E1', 'KKKs_E2', 'KK_KKKs', 'KKP_KKKs', 'KKPP_KKPase', 'KKP_KKPase',
    'K_KKPP', 'KP_KKPP', 'KPP_KPase', 'KP_KPase',
]


def mapk_cascade(n_inst: int = 256, seed: int = 5, variant: bool = False,
                 scale: float = 1.0) -> Tuple[Model, Property]:
    """Three-tier phosphorylation cascade (22 species, 30 reactions).

    Ten enzymatic steps E + S <-> ES -> E + P: tier 1 activates KKK by E1 and
    deactivates it by E2; tier 2 double-phosphorylates KK by KKK* and
    dephosphorylates it by KKPase; tier 3 does the same for K by KK-PP and
    KPase.  Every complex dissociates at 0.1 and converts at kcat (0.8 and
    0.3 in tier 1, 1.0 below); the binding constants give Michaelis constants
    (koff + kcat) / kon of 90 and 65 (tier 1), 2000 (tier 2) and 4000
    (tier 3) molecules.  The initial state is a pulse: all 900 KKK
    molecules active, a weak activator (E1 = 2) against E2 = 100, KK = 2400,
    K = 6000 (counts reach about 6000), KKPase = 250, KPase = 800, so that
    KPP rises to about 2000 near t = 40 and falls back within tens of time
    units, and a trajectory runs about 1.4e5 events before its verdict is
    fixed.  Rate constants are these base values times a per-instance
    log-uniform factor in [0.8, 1.25].  ``scale`` multiplies the KKK, KK and
    K counts.  The property is (KPP<500) U[0,200] (KPP>=2000 & F[0,50]
    KPP<500); ``variant=True`` replaces the left operand by KPP<2000.
    """
    sp = MAPK_SPECIES
    koff = 0.1
    steps = [  # (enzyme, substrate, product, complex, Michaelis constant, kcat)
        ('E1', 'KKK', 'KKKs', 'KKK_E1', 90.0, 0.8),
        ('E2', 'KKKs', 'KKK', 'KKKs_E2', 65.0, 0.3),
        ('KKKs', 'KK', 'KKP', 'KK_KKKs', 2000.0, 1.0),
        ('KKKs', 'KKP', 'KKPP', 'KKP_KKKs', 2000.0, 1.0),
        ('KKPase', 'KKPP', 'KKP', 'KKPP_KKPase', 2000.0, 1.0),
        ('KKPase', 'KKP', 'KK', 'KKP_KKPase', 2000.0, 1.0),
        ('KKPP', 'K', 'KP', 'K_KKPP', 4000.0, 1.0),
        ('KKPP', 'KP', 'KPP', 'KP_KKPP', 4000.0, 1.0),
        ('KPase', 'KPP', 'KP', 'KPP_KPase', 4000.0, 1.0),
        ('KPase', 'KP', 'K', 'KP_KPase', 4000.0, 1.0),
    ]
    reactions, base = [], []
    for enz, sub, prod, cplx, km, kcat in steps:
        reactions.append(([enz, sub], [cplx]))
        base.append((koff + kcat) / km)
        reactions.append(([cplx], [enz, sub]))
        base.append(koff)
        reactions.append(([cplx], [enz, prod]))
        base.append(kcat)
    reac, st = _net(sp, reactions)
    init = dict(KKKs=900, E1=2, E2=100, KK=2400, KKPase=250, K=6000, KPase=800)
    x0 = np.array([int(round(init.get(s, 0) * (scale if s in ('KK', 'K', 'KKKs') else 1.0)))
                   for s in sp], np.int32)
    rng = np.random.default_rng(seed)
    fac = np.exp(rng.uniform(math.log(0.8), math.log(1.25), size=(n_inst, len(base))))
    rates = np.asarray(base)[None, :] * fac
    m = Model('mapk_variant' if variant else 'mapk', sp, reac, st, rates, np.tile(x0, (n_inst, 1)))
    left_bound = 2000 if variant else 500
    p = Property([atom(sp, 'KPP', '<', left_bound), atom(sp, 'KPP', '>=', 2000),
                  atom(sp, 'KPP', '<', 500)],
                 ('U', 0.0, 200.0, ('atom', 0), ('and', ('atom', 1), ('F', 0.0, 50.0, ('atom', 2)))),
                 f'(KPP<{left_bound}) U[0,200] (KPP>=2000 & F[0,50] KPP<500)')
    return m, p


def formula_atoms(f) -> set:
    """Atom indices used by a formula tree."""
    if f[0] == 'atom':
        return {f[1]}
    out = set()
    for c in f[1:]:
        if isinstance(c, tuple):
            out |= formula_atoms(c)
    return out
