"""The kernels' linear atoms (atom_bit in smc_device.cuh, compiled for the
host, reading an instance table built by the library's build_blob): on
random states, every atom's bit equals the FP64 comparison (double)L <op> b
of its linear form L = sum_i coef_i x_i, for single-term atoms (the fast
path) and multi-term ones, all six operators, integer and fractional
bounds."""
import os
import random
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')
OPS = ['<', '<=', '>=', '>', '==', '!=']


def test_device_linear_atoms(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    exe = str(tmp_path / 'atom_device_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(ROOT, 'tests'), '-I', os.path.join(CUDA, 'include'),
                    os.path.join(ROOT, 'tests', 'atom_device_check.cpp'), os.path.join(CSRC, 'smc_compile.cpp'),
                    '-o', exe, '-lm'], check=True)
    rng = random.Random(9)
    for trial in range(40):
        S = rng.randint(1, 12)
        atoms = []
        for a in range(6):
            coef = [0] * S
            for i in rng.sample(range(S), rng.randint(1, min(S, 4))):
                coef[i] = rng.choice([1, 1, 2, -1, -3, 5])
            atoms.append((rng.choice(OPS), rng.choice([0.0, 1.0, 7.0, -2.0, 2.5, 130.0, rng.randint(-50, 300)]),
                          coef))
        states = [[rng.choice([0, 1, 2, 3, 7, rng.randint(0, 300)]) for _ in range(S)] for _ in range(200)]
        lines = [f'{S} {len(atoms)}']
        lines += [f'{OPS.index(op)} {b!r} ' + ' '.join(map(str, c)) for op, b, c in atoms]
        lines += [' '.join(map(str, x)) for x in states]
        r = subprocess.run([exe], input='\n'.join(lines) + '\n', capture_output=True, text=True, timeout=60)
        assert r.returncode == 0, r.stdout + r.stderr
        got = [int(v) for v in r.stdout.split()]
        assert len(got) == len(states)
        for x, bits in zip(states, got):
            for a, (op, b, c) in enumerate(atoms):
                L = float(np.dot(c, x))
                want = {'<': L < b, '<=': L <= b, '>=': L >= b, '>': L > b, '==': L == b, '!=': L != b}[op]
                assert bool((bits >> a) & 1) == want, (S, atoms[a], x)
