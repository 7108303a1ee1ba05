"""The compiled BLTLc monitor on the host: the device code the SSA kernels
step (smc_device.cuh), compiled for the host by tests/monitor_host.cpp and
driven over exhaustive tiny paths (all count sequences of length <= 5 over
{0..3}, entry times on and off the window bounds), must fix the same
verdict at the same point as the oracle's trace semantics, for every
formula of the oracle's monitor tests (nested F / G, until with windows,
boolean combinations, Next).  The GPU test of the replay kernel runs the
same comparison on the device.  The same paths also go through the trace
monitor (smc_nest.h) for every formula, and it alone serves the formulas
nested beyond the unit monitor's shapes; and through the trace monitor
with its memo, evaluated at every knowledge point in the SSA's order, or at
a pseudo-random subset of them as the kernel's deferred checks take them
(the memo's results equal to the plain evaluation at each point), on the
tiny paths and on long ones whose windows hold many positions."""
import math
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

import workloads
from paper_0912_2551_gb300 import postfix
from paper_0912_2551_gb300._native import OP
from tests.test_gpu_parity import _oracle_decision_point
from tests.test_oracle_monitor import FORMULAS, _atoms, _paths

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')


@pytest.fixture(scope='module')
def exe(tmp_path_factory):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    out = str(tmp_path_factory.mktemp('mon') / 'monitor_host')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(CUDA, 'include'), os.path.join(ROOT, 'tests', 'monitor_host.cpp'),
                    os.path.join(CSRC, 'smc_compile.cpp'), '-o', out], check=True)
    return out


def _run(exe, prop, paths, mode):
    S = 1
    lines = [f'{S} {len(prop.atoms)} {len(postfix(prop.formula))}']
    for a in prop.atoms:
        lines.append(f'{OP[a.op]} {a.bound!r} ' + ' '.join(str(int(c)) for c in a.coef))
    for kind, arg, lo, hi in postfix(prop.formula):
        lines.append(f'{kind} {arg} {lo!r} {hi!r}')
    lines.append(str(len(paths)))
    for xs, ts, tmin, closed in paths:
        lines.append(f'{len(ts)} {int(closed)} {"inf" if math.isinf(tmin) else repr(float(tmin))}')
        lines.append(' '.join(str(int(v)) for v in xs))
        lines.append(' '.join(repr(float(v)) for v in ts))
    args = [exe] + ([mode] if mode != 'library' else [])
    r = subprocess.run(args, input='\n'.join(lines) + '\n', capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    out = [tuple(int(w) for w in ln.split()) for ln in r.stdout.splitlines()]
    assert len(out) == len(paths)
    return out


@pytest.mark.parametrize('fi', range(len(FORMULAS)))
def test_trace_monitor_memo_on_long_paths(exe, orc, fi):
    # 40-90 positions, steps of 0-0.5 time units: a [0, 3] window holds a
    # dozen positions or more, so nested windows share most of their cells
    prop = workloads.Property(_atoms(), FORMULAS[fi])
    rng = random.Random(7000 + fi)
    paths = []
    for _ in range(24):
        n = rng.randint(40, 90)
        xs, ts = [rng.randrange(4)], [0.0]
        for _ in range(n - 1):
            xs.append(min(3, max(0, xs[-1] + rng.choice([-1, 1, 1, -1, 0]))))
            ts.append(ts[-1] + rng.choice([0.0, 0.25, 0.5, 0.5 * rng.random()]))
        closed = rng.random() < 0.3
        tmin = math.inf if closed else ts[-1] + rng.choice([0.0, 0.5, 3.0])
        paths.append((np.asarray(xs), np.asarray(ts, float), tmin, closed))
    out = _run(exe, prop, paths, 'memo')
    assert _run(exe, prop, paths, 'memo_sparse') == out
    for (v, q), (xs, ts, tmin, closed) in zip(out[:8], paths[:8]):
        ov, oq = _oracle_decision_point(orc, prop, 1, xs, ts, tmin, closed)
        assert (v, q) == ({0: 1, 1: 2, 2: 0}[ov], oq), (FORMULAS[fi], v, q, ov, oq)


@pytest.mark.parametrize('mode', ['library', 'nest', 'memo', 'memo_sparse'])
@pytest.mark.parametrize('fi', range(len(FORMULAS)))
def test_monitor_matches_oracle_on_tiny_paths(exe, orc, fi, mode):
    # library: the unit monitor for the formulas of its fragment, the trace
    # monitor for the rest; nest: the trace monitor for every formula; memo:
    # the same with its memo, at every knowledge point in turn
    prop = workloads.Property(_atoms(), FORMULAS[fi])
    S = 1
    rng = random.Random(1000 + fi)
    paths = []
    for xs, ts in _paths(rng, 400):
        closed = rng.random() < 0.3
        tmin = math.inf if closed else ts[-1] + rng.choice([0.0, 0.5, 1.0, 3.0])
        paths.append((np.asarray(xs), np.asarray(ts, float), tmin, closed))
    out = _run(exe, prop, paths, mode)
    for (v, q), (xs, ts, tmin, closed) in zip(out, paths):
        ov, oq = _oracle_decision_point(orc, prop, S, xs, ts, tmin, closed)
        want = {0: 1, 1: 2, 2: 0}[ov]
        assert (v, q) == (want, oq), (FORMULAS[fi], xs.tolist(), ts.tolist(), tmin, closed, v, q, ov, oq)
