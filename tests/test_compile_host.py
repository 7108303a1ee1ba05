"""The library's host-side formula compiler and atom helpers
(paper_0912_2551_gb300/csrc/smc_compile.cpp), compiled for the host and
checked by tests/compile_check.cpp: atom thresholds by brute force against
the FP64 comparison, atom-program validation and evaluation, postfix
parsing, the monitor units of the workloads' formulas, the three-valued
verdict tables of boolean combinations against Kleene's logic, and the
rejection of every formula outside the monitorable fragment."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')


def test_formula_compiler(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    exe = str(tmp_path / 'compile_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(CUDA, 'include'), os.path.join(ROOT, 'tests', 'compile_check.cpp'),
                    os.path.join(CSRC, 'smc_compile.cpp'), '-o', exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith('ok'), r.stdout + r.stderr
