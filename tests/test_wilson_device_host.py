"""The Wilson interval the kernels compute at the end of a launch (Eq. 4,
wilson_eq4 in smc_device.cuh, compiled for the host) against the oracle's
Eq. 4: the estimate exactly, the bounds to 1e-12 relative, over counts
from 0/n to n/n and n from 1 to 10^9, at 90%, 95% and 99%."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import wilson

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')


def test_device_wilson_matches_oracle(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    exe = str(tmp_path / 'wilson_device_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(ROOT, 'tests'), '-I', os.path.join(CUDA, 'include'),
                    os.path.join(ROOT, 'tests', 'wilson_device_check.cpp'), '-o', exe, '-lm'], check=True)
    rng = np.random.default_rng(7)
    cases = []
    for conf in (0.90, 0.95, 0.99):
        z = wilson.z_value(conf)
        for n in (1, 2, 3, 10, 127, 2648, 10_000, 1_000_000, 10**9):
            for yes in sorted({0, 1, n // 2, n - 1, n, int(rng.integers(0, n + 1)), int(0.0912186 * n)}):
                if 0 <= yes <= n:
                    cases.append((yes, n, z, conf))
    inp = '\n'.join(f'{y} {n} {z!r}' for y, n, z, _ in cases) + '\n'
    r = subprocess.run([exe], input=inp, capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stderr
    rows = [[float(v) for v in ln.split()] for ln in r.stdout.splitlines()]
    assert len(rows) == len(cases)
    for (yes, n, z, conf), (p, lo, hi) in zip(cases, rows):
        op, olo, ohi = wilson.wilson_interval(yes, n, conf)
        assert p == op == yes / n
        assert abs(lo - olo) <= 1e-12 * max(abs(olo), 1e-300)
        assert abs(hi - ohi) <= 1e-12 * abs(ohi)
        if yes == 0:
            assert lo == 0.0
        if yes == n:
            assert hi == 1.0
