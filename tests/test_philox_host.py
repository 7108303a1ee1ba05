"""The kernels' Philox4x32-10 and uniform maps (smc_device.cuh, compiled
for the host) against the oracle's independent implementation on 10^8
counter blocks, bit for bit (tests/philox_check.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')


def test_philox_kernel_equals_oracle_on_1e8_blocks(tmp_path):
    gxx, gcc = shutil.which('g++'), shutil.which('gcc')
    if gxx is None or gcc is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no compilers or CUDA headers')
    obj = str(tmp_path / 'oracle.o')
    subprocess.run([gcc, '-O2', '-ffp-contract=off', '-c', os.path.join(ROOT, 'oracle', 'smc_oracle.c'), '-o', obj],
                   check=True)
    exe = str(tmp_path / 'philox_check')
    subprocess.run([gxx, '-O2', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(ROOT, 'tests'), '-I', os.path.join(CUDA, 'include'),
                    os.path.join(ROOT, 'tests', 'philox_check.cpp'), obj, '-o', exe, '-lm', '-lpthread'], check=True)
    r = subprocess.run([exe, '100000000'], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    kv = dict(f.split('=') for f in r.stdout.split())
    assert int(kv['blocks']) == 100_000_000
    assert kv['mismatches'] == '0' and kv['u52'] == '0' and kv['u23'] == '0'
