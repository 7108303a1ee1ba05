"""The model-specialized kernels' generated code (jit_model_header in
paper_0912_2551_gb300/csrc/smc_jit.cpp), evaluated on the host: the header
the library writes for a network is compiled with the CUDA intrinsics it
calls replaced by the IEEE-754 operations they denote, and on random states
its FP64 propensity prefix sums must equal, bit for bit, the arithmetic the
FP64 path is defined by: a_k = c_k * (double)h_k with h the exact
mass-action count (h = 1, x_a, x_a x_b or x_a (x_a - 1) / 2), then each
rate-law factor in order (xn = x, times x (n - 1) more times, num = a0 + a1
xn, den = b0 + b1 xn, a = a * (num / den)), summed left to right.  The
positive-propensity mask, the state updates x += v_j and the atom bits are
checked too; the FP32 (mixed) sums agree to FP32 rounding."""
import math
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
BUILD = os.path.join(ROOT, 'paper_0912_2551_gb300', '_build')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')
INT64_MAX = (1 << 63) - 1
INT64_MIN = -(1 << 63)


@pytest.fixture(scope='module')
def dumper(tmp_path_factory):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    from paper_0912_2551_gb300 import build as native_build
    native_build.build()  # the embedded kernel sources smc_jit.cpp includes
    d = tmp_path_factory.mktemp('jit')
    exe = str(d / 'jit_header_dump')
    subprocess.run([gxx, '-O1', '-std=c++17', '-I', CSRC, '-I', BUILD, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(CUDA, 'include'), os.path.join(ROOT, 'tests', 'jit_header_dump.cpp'),
                    os.path.join(CSRC, 'smc_jit.cpp'), os.path.join(CSRC, 'smc_compile.cpp'), '-o', exe,
                    '-L', os.path.join(CUDA, 'lib64'), '-lcudart', '-ldl'], check=True)
    return gxx, exe, d


def _threshold(op, b):
    """lo, hi, neg with L <op> b  <=>  (lo <= L <= hi) xor neg over integers."""
    if op == '<':
        return INT64_MIN, math.ceil(b) - 1, 0
    if op == '<=':
        return INT64_MIN, math.floor(b), 0
    if op == '>=':
        return math.ceil(b), INT64_MAX, 0
    if op == '>':
        return math.floor(b) + 1, INT64_MAX, 0
    lo, hi = (int(b), int(b)) if float(b).is_integer() else (1, 0)
    return lo, hi, int(op == '!=')


def _header(dumper, model, atoms, name):
    gxx, exe, d = dumper
    S, R = model.n_species, model.n_reactions
    parts = [f'{S} {R} {len(atoms)} {len(model.factors)}', ' '.join(map(str, model.reactants.ravel())),
             ' '.join(map(str, model.stoich.ravel()))]
    for a in atoms:
        lo, hi, neg = _threshold(a.op, a.bound)
        parts.append(' '.join(map(str, a.coef)) + f' {lo} {hi} {neg}')
    for f in model.factors:
        parts.append(' '.join(map(str, f[:3])) + ' ' + ' '.join(repr(float(v)) for v in f[3:]))
    env = dict(os.environ, LD_LIBRARY_PATH=os.path.join(CUDA, 'lib64') + ':' + os.environ.get('LD_LIBRARY_PATH', ''))
    r = subprocess.run([exe], input='\n'.join(parts) + '\n', capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0, r.stderr
    inc = d / name
    inc.mkdir()
    (inc / 'jit_model.h').write_text(r.stdout)
    ev = str(inc / 'eval')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', str(inc), '-I', CSRC,
                    os.path.join(ROOT, 'tests', 'jit_host_eval.cpp'), '-o', ev], check=True)
    return ev


def _expected_prefix(model, rates, x):
    acc, pre = None, []
    for k in range(model.n_reactions):
        ra, rb = (int(v) for v in model.reactants[k])
        if ra < 0 and rb < 0:
            h = 1
        elif ra < 0 or rb < 0:
            h = int(x[max(ra, rb)])
        elif ra == rb:
            h = int(x[ra]) * (int(x[ra]) - 1) // 2
        else:
            h = int(x[ra]) * int(x[rb])
        a = float(rates[k]) * float(h)
        for (kk, m, n, a0, a1, b0, b1) in model.factors:
            if kk != k:
                continue
            xv = float(x[m])
            xn = xv
            for _ in range(n - 1):
                xn = xn * xv
            a = a * ((a0 + a1 * xn) / (b0 + b1 * xn))
        acc = a if acc is None else acc + a
        pre.append(acc)
    return pre


def _check(ev, model, atoms, n_states=300, seed=0):
    S, R = model.n_species, model.n_reactions
    rng = np.random.default_rng(seed)
    rates = model.rates[0]
    states = rng.integers(0, 60, size=(n_states, S))
    states[:n_states // 4] = rng.integers(0, 3, size=(n_states // 4, S))  # many zeros and ones
    states[n_states // 4:n_states // 2] = rng.integers(0, 5000, size=(n_states // 4, S))
    inp = ' '.join(repr(float(c)) for c in rates) + '\n' + '\n'.join(' '.join(map(str, s)) for s in states) + '\n'
    r = subprocess.run([ev], input=inp, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    lines = r.stdout.splitlines()
    per = 3 + R
    assert len(lines) == per * n_states
    for i, x in enumerate(states):
        block = lines[i * per:(i + 1) * per]
        got = [struct.unpack('<d', bytes.fromhex(w)[::-1])[0] for w in block[0].split()[1:]]
        want = _expected_prefix(model, rates, x)
        assert all(struct.pack('<d', g) == struct.pack('<d', w) for g, w in zip(got, want)), (x, got, want)
        m = block[1].split()
        pos, posf = int(m[1]), int(m[2])
        # positive-propensity mask: bit k iff a_k > 0
        ak = [_expected_prefix_term(model, rates, x, k) for k in range(R)]
        want_pos = sum(1 << k for k in range(R) if ak[k] > 0)
        assert pos == want_pos and posf == want_pos
        mixed = [float(v) for v in m[3:]]
        for g, w in zip(mixed, want):
            assert abs(g - w) <= 2e-6 * abs(w) * R + 1e-30
        bits = int(block[2].split()[1])
        for a_i, a in enumerate(atoms):
            L = int(np.dot(a.coef.astype(np.int64), x))
            b = a.bound
            want_b = {'<': L < b, '<=': L <= b, '>=': L >= b, '>': L > b, '==': L == b, '!=': L != b}[a.op]
            assert bool((bits >> a_i) & 1) == want_b
        for j in range(R):
            y = np.array([int(v) for v in block[3 + j].split()[1:]])
            assert np.array_equal(y, x + model.stoich[j])


def _expected_prefix_term(model, rates, x, k):
    """a_k alone, by the same arithmetic."""
    pre = _expected_prefix(_OneReaction(model, k), rates[k:k + 1], x)
    return pre[0]


class _OneReaction:
    def __init__(self, model, k):
        self.n_reactions = 1
        self.reactants = model.reactants[k:k + 1]
        self.factors = [(0,) + tuple(f[1:]) for f in model.factors if f[0] == k]


def _cases():
    yield 'lotka_volterra', workloads.lotka_volterra()
    yield 'immigration_death', workloads.immigration_death()
    yield 'dimerisation', workloads.dimerisation()
    yield 'autorepressor', workloads.autorepressor()
    yield 'mm_degradation', workloads.mm_degradation()
    yield 'factor_chain', workloads.factor_chain()
    yield 'cascade', workloads.mapk_cascade(n_inst=1)


@pytest.mark.parametrize('name', ['lotka_volterra', 'immigration_death', 'dimerisation', 'autorepressor',
                                  'mm_degradation', 'factor_chain', 'cascade'])
def test_generated_code_matches_the_fp64_definition(dumper, name):
    model, prop = dict(_cases())[name]
    atoms = [a for a in prop.atoms if a.lhs is None]
    ev = _header(dumper, model, atoms, name)
    _check(ev, model, atoms)


def test_generated_code_on_random_networks(dumper):
    batch = workloads.random_networks(n_inst=60, seed=11)
    done = 0
    for i, (model, prop) in enumerate(zip(batch.models, batch.properties)):
        if model.n_species > 32 or model.n_reactions > 32:
            continue
        ev = _header(dumper, model, prop.atoms, f'rn{i}')
        _check(ev, model, prop.atoms, n_states=60, seed=i)
        done += 1
        if done == 6:
            break
    assert done == 6
