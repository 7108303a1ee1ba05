"""The kernels' arithmetic atoms (BLTLc's val <| val, Sec. 3.1; eval_expr /
expr_atom_bit in smc_device.cuh, compiled for the host): on random postfix
programs and states, including division by zero and square roots of
negative values, each side's value equals bit for bit the program
evaluated by its definition (each operation rounded once, sqrt correctly
rounded, integer powers by repeated multiplication), and the atom's truth
equals the oracle's."""
import math
import os
import random
import shutil
import struct
import subprocess

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')
KIND = {'x': 0, 'c': 1, '+': 2, '-': 3, '*': 4, '/': 5, 'sqrt': 6, 'pow': 7}
OPS = {'<': 0, '<=': 1, '>=': 2, '>': 3, '==': 4, '!=': 5}


def _program(rng, S):
    toks, depth = [], 0
    n = rng.randint(1, 12)
    while len(toks) < n or depth != 1:
        choices = []
        if depth < 6 and len(toks) < 20:
            choices += ['x', 'c']
        if depth >= 2:
            choices += ['+', '-', '*', '/']
        if depth >= 1:
            choices += ['sqrt', 'pow']
        k = rng.choice(choices)
        if k == 'x':
            toks.append(('x', rng.randrange(S)))
            depth += 1
        elif k == 'c':
            toks.append(('c', rng.choice([0.0, 1.0, -1.0, 2.5, -3.0, 0.1, 1e3, rng.uniform(-10, 10)])))
            depth += 1
        elif k == 'pow':
            toks.append(('pow', rng.randint(0, 5)))
        elif k == 'sqrt':
            toks.append(('sqrt',))
        else:
            toks.append((k,))
            depth -= 1
    return toks


def _evaluate(toks, x):
    st = []
    for t in toks:
        k = t[0]
        if k == 'x':
            st.append(float(x[t[1]]))
        elif k == 'c':
            st.append(float(t[1]))
        elif k == 'sqrt':
            a = st.pop()
            st.append(math.sqrt(a) if a >= 0 else (a if math.isnan(a) else math.nan))
        elif k == 'pow':
            a = st.pop()
            r = 1.0
            if t[1] > 0:
                r = a
                for _ in range(t[1] - 1):
                    r = r * a
            st.append(r)
        else:
            b, a = st.pop(), st.pop()
            if k == '+':
                st.append(a + b)
            elif k == '-':
                st.append(a - b)
            elif k == '*':
                st.append(a * b)
            else:
                st.append(a / b if b != 0 else (math.nan if a == 0 or math.isnan(a) else math.copysign(math.inf, a) * math.copysign(1.0, b)))
    assert len(st) == 1
    return st[0]


def _bits(v):
    return struct.unpack('<Q', struct.pack('<d', v))[0]


def test_device_arithmetic_atoms(tmp_path, orc):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    exe = str(tmp_path / 'expr_device_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(ROOT, 'tests'), '-I', os.path.join(CUDA, 'include'),
                    os.path.join(ROOT, 'tests', 'expr_device_check.cpp'), '-o', exe, '-lm'], check=True)
    rng = random.Random(5)
    S = 3
    cases = []
    for _ in range(1500):
        lhs, rhs = _program(rng, S), _program(rng, S)
        op = rng.choice(list(OPS))
        x = [rng.choice([0, 0, 1, 2, 3, 7, 50, rng.randint(0, 10_000)]) for _ in range(S)]
        cases.append((lhs, op, rhs, x))
    lines = [str(S)]
    for lhs, op, rhs, x in cases:
        lines.append(f'{OPS[op]} {len(lhs)} {len(rhs)}')
        for t in lhs + rhs:
            k = KIND[t[0]]
            lines.append(f'{k} {t[1] if k in (0, 7) else 0} {float(t[1]) if k == 1 else 0.0!r}')
        lines.append(' '.join(map(str, x)))
    r = subprocess.run([exe], input='\n'.join(lines) + '\n', capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = r.stdout.splitlines()
    assert len(out) == len(cases)
    sp = ['a', 'b', 'c']
    nan_cases = 0
    for (lhs, op, rhs, x), line in zip(cases, out):
        hl, hr, bit = line.split()
        for h, prog in ((hl, lhs), (hr, rhs)):
            want = _evaluate(prog, x)
            got = struct.unpack('<d', struct.pack('<Q', int(h, 16)))[0]
            if math.isnan(want):
                nan_cases += 1
                assert math.isnan(got), (prog, x, got)
            else:
                assert int(h, 16) == _bits(want), (prog, x, got, want)
        atom = workloads.Atom(np.zeros(S, np.int32), op, 0.0, lhs, rhs)
        prop = workloads.Property([atom], ('atom', 0))
        ov = orc.eval_prefix(prop, S, np.asarray([x]), np.asarray([0.0]), math.inf, True)
        assert ov in (0, 1) and int(bit) == ov, (lhs, op, rhs, x, bit, ov)
    assert nan_cases > 10  # the undefined operations were exercised
