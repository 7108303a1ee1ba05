"""The per-instance table the SSA kernels read (build_blob in
paper_0912_2551_gb300/csrc/smc_compile.cpp), built on the host by
tests/blob_check.cpp and decoded here section by section against the
network it came from: rate constants (FP64 and FP32), propensity words
(the word's formula x_ra (x_rb - homo) >> homo, with a constant-1 column,
equals the mass-action combinatorics on random states), the stoichiometry
CSR and dense rows, the dependency CSR (recomputed here from the
reactants and the rate-law factors' species), atom terms, masks and
thresholds (brute force against the FP64 comparison), initial counts and
rate-law factors."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')
OPS = {'<': 0, '<=': 1, '>=': 2, '>': 3, '==': 4, '!=': 5}
(BH_S, BH_R, BH_NA, BH_WORDS, BH_RATE_D, BH_RATE_F, BH_REAC, BH_ST_PTR, BH_ST, BH_DEP_PTR, BH_DEP, BH_AMASK,
 BH_ATERM_PTR, BH_ATERM, BH_X0, BH_ATOM, BH_DENSE, BH_FACT_PTR, BH_FACT, BH_FACT_D, BH_FACT_F) = range(21)


@pytest.fixture(scope='module')
def exe(tmp_path_factory):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    out = str(tmp_path_factory.mktemp('blob') / 'blob_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(CUDA, 'include'), os.path.join(ROOT, 'tests', 'blob_check.cpp'),
                    os.path.join(CSRC, 'smc_compile.cpp'), '-o', out], check=True)
    return out


def _build(exe, model, atoms):
    S, R = model.n_species, model.n_reactions
    parts = [f'{S} {R} {len(atoms)} {len(model.factors)}',
             ' '.join(str(int(v)) for v in model.reactants.ravel()),
             ' '.join(str(int(v)) for v in model.stoich.ravel()),
             ' '.join(repr(float(v)) for v in model.rates[0]),
             ' '.join(str(int(v)) for v in model.x0[0])]
    for a in atoms:
        parts.append(f'{OPS[a.op]} {a.bound!r} ' + ' '.join(str(int(c)) for c in a.coef))
    for (k, m, n, a0, a1, b0, b1) in model.factors:
        parts.append(f'{k} {m} {n} {a0!r} {a1!r} {b0!r} {b1!r}')
    r = subprocess.run([exe], input='\n'.join(parts) + '\n', capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.array([int(w) for w in r.stdout.split()], dtype=np.uint64).astype(np.uint32)


def _i32(w):
    return np.asarray(w, np.uint32).view(np.int32)


def _f64(blob, off, n):
    return np.frombuffer(blob[off:off + 2 * n].tobytes(), dtype='<f8')


def _mass_action_h(reactants, x):
    a, b = reactants
    if a < 0 and b < 0:
        return 1
    if a < 0 or b < 0:
        return int(x[max(a, b)])
    if a == b:
        return int(x[a]) * (int(x[a]) - 1) // 2
    return int(x[a]) * int(x[b])


def _check(blob, model, atoms):
    S, R, NA = model.n_species, model.n_reactions, len(atoms)
    st = model.stoich.astype(np.int64)
    assert (blob[BH_S], blob[BH_R], blob[BH_NA]) == (S, R, NA)
    assert blob[BH_WORDS] == len(blob) and len(blob) % 4 == 0
    order = [BH_RATE_D, BH_RATE_F, BH_REAC, BH_ST_PTR, BH_ST, BH_DEP_PTR, BH_DEP, BH_AMASK, BH_ATERM_PTR, BH_ATERM]
    offs = [int(blob[h]) for h in order]
    assert offs == sorted(offs) and all(o % 2 == 0 and o < len(blob) for o in offs)
    # rate constants
    o = int(blob[BH_RATE_D])
    assert np.array_equal(_f64(blob, o, R), model.rates[0])
    o = int(blob[BH_RATE_F])
    assert np.array_equal(blob[o:o + R].view(np.float32), model.rates[0].astype(np.float32))
    # propensity words
    o = int(blob[BH_REAC])
    pw = blob[o:o + R].astype(np.int64)
    fact_reactions = {f[0] for f in model.factors}
    rng = np.random.default_rng(S * 131 + R)
    for k in range(R):
        assert pw[k] & 0xFF == k
        assert bool(pw[k] & (1 << 25)) == (k in fact_reactions)
        ra, rb, homo = (pw[k] >> 8) & 0xFF, (pw[k] >> 16) & 0xFF, (pw[k] >> 24) & 1
        for _ in range(20):
            x = np.append(rng.integers(0, 50, S), 1)  # species index S: the constant-1 column
            assert (int(x[ra]) * (int(x[rb]) - homo)) >> homo == _mass_action_h(model.reactants[k], x)
    # stoichiometry CSR
    p0, o = int(blob[BH_ST_PTR]), int(blob[BH_ST])
    ptr = blob[p0:p0 + R + 1].astype(np.int64)
    dense = np.zeros((R, S), np.int64)
    for j in range(R):
        for w in _i32(blob[o + ptr[j]:o + ptr[j + 1]]):
            dense[j, w & 0xFF] = w >> 8
    assert np.array_equal(dense, st)
    # dependency CSR: k in dep(j) iff a_k reads a species j changes
    p0, o = int(blob[BH_DEP_PTR]), int(blob[BH_DEP])
    ptr = blob[p0:p0 + R + 1].astype(np.int64)
    reads = [set(int(s) for s in model.reactants[k] if s >= 0) | {f[1] for f in model.factors if f[0] == k}
             for k in range(R)]
    for j in range(R):
        words = blob[o + ptr[j]:o + ptr[j + 1]].astype(np.int64)
        changed = set(np.nonzero(st[j])[0].tolist())
        assert sorted(int(w) & 0xFF for w in words) == [k for k in range(R) if reads[k] & changed]
        assert all(w == pw[int(w) & 0xFF] for w in words)
    # atoms: masks, terms, records
    o = int(blob[BH_AMASK])
    amask = blob[o:o + R]
    p0, o = int(blob[BH_ATERM_PTR]), int(blob[BH_ATERM])
    ptr = blob[p0:p0 + NA + 1].astype(np.int64)
    rec = int(blob[BH_ATOM])
    for a, at in enumerate(atoms):
        coef = at.coef.astype(np.int64)
        for j in range(R):
            assert bool((amask[j] >> a) & 1) == bool(coef @ st[j] != 0)
        terms = np.zeros(S, np.int64)
        for w in _i32(blob[o + ptr[a]:o + ptr[a + 1]]):
            terms[w & 0xFF] = w >> 8
        assert np.array_equal(terms, coef)
        r = blob[rec + 6 * a:rec + 6 * a + 6]
        single = np.count_nonzero(coef) == 1
        assert (r[0] != 0xFFFFFFFF) == single
        neg = bool(r[1])
        lo = int(np.array([r[2], r[3]], np.uint32).view(np.int64)[0])
        hi = int(np.array([r[4], r[5]], np.uint32).view(np.int64)[0])
        b = float(at.bound)
        for L in range(-50, 400):
            want = {'<': L < b, '<=': L <= b, '>=': L >= b, '>': L > b, '==': L == b, '!=': L != b}[at.op]
            assert ((lo <= L <= hi) != neg) == want
    # initial counts
    o = int(blob[BH_X0])
    assert np.array_equal(_i32(blob[o:o + S]), model.x0[0])
    # dense int8 rows of small networks
    small = S <= 8 and R <= 8 and np.abs(st).max() <= 127
    assert (blob[BH_DENSE] != 0) == small
    if small:
        o = int(blob[BH_DENSE])
        rows = blob[o:o + 2 * R].view(np.int8).reshape(R, 8)[:, :S]
        assert np.array_equal(rows.astype(np.int64), st)
    # rate-law factors, in order within each reaction
    if model.factors:
        p0, o = int(blob[BH_FACT_PTR]), int(blob[BH_FACT])
        ptr = blob[p0:p0 + R + 1].astype(np.int64)
        od, of = int(blob[BH_FACT_D]), int(blob[BH_FACT_F])
        for k in range(R):
            mine = [f for f in model.factors if f[0] == k]
            assert ptr[k + 1] - ptr[k] == len(mine)
            for q, f in zip(range(ptr[k], ptr[k + 1]), mine):
                assert blob[o + q] == f[1] | (f[2] << 8)
                assert np.array_equal(_f64(blob, od + 8 * q, 4), np.array(f[3:], np.float64))
                assert np.array_equal(blob[of + 4 * q:of + 4 * q + 4].view(np.float32),
                                      np.array(f[3:], np.float32))
    else:
        assert blob[BH_FACT_PTR] == 0


def _cases():
    yield 'lotka_volterra', *workloads.lotka_volterra()
    yield 'immigration_death', *workloads.immigration_death()
    yield 'dimerisation', *workloads.dimerisation()
    yield 'autorepressor', *workloads.autorepressor()
    yield 'factor_chain', *workloads.factor_chain()
    m, p = workloads.mapk_cascade(n_inst=1)
    yield 'cascade', m, p


@pytest.mark.parametrize('name', ['lotka_volterra', 'immigration_death', 'dimerisation', 'autorepressor',
                                  'factor_chain', 'cascade'])
def test_blob_of_workload(exe, name):
    for nm, model, prop in _cases():
        if nm == name:
            _check(_build(exe, model, prop.atoms), model, prop.atoms)


def test_blob_of_random_networks(exe):
    batch = workloads.random_networks(n_inst=24)
    for model, prop in zip(batch.models, batch.properties):
        _check(_build(exe, model, prop.atoms), model, prop.atoms)
