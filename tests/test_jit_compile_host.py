"""The model-specialized kernels compile for sm_103a (NVRTC, no GPU needed):
tests/jit_compile_check.cpp generates the model header for a small network,
one with a rate-law factor, one with an arithmetic atom and a medium one
(22 species, 30 reactions), and compiles the kernels through the library's
own code path; without a GPU only the final load of the cubin fails."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')
BUILD = os.path.join(ROOT, 'paper_0912_2551_gb300', '_build')
CUDA = os.environ.get('CUDA_HOME', '/usr/local/cuda')


def test_specialized_kernels_compile(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None or not os.path.exists(os.path.join(CUDA, 'include', 'cuda_runtime.h')):
        pytest.skip('no g++ or CUDA headers')
    from paper_0912_2551_gb300 import build as native_build
    native_build.build()  # writes the embedded kernel sources the library compiles
    exe = str(tmp_path / 'jit_compile_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-I', CSRC, '-I', BUILD, '-I', os.path.join(ROOT, 'include'),
                    '-I', os.path.join(CUDA, 'include'), os.path.join(ROOT, 'tests', 'jit_compile_check.cpp'),
                    os.path.join(CSRC, 'smc_jit.cpp'), os.path.join(CSRC, 'smc_compile.cpp'), '-o', exe,
                    '-L', os.path.join(CUDA, 'lib64'), '-lcudart', '-ldl'], check=True)
    env = dict(os.environ, LD_LIBRARY_PATH=os.path.join(CUDA, 'lib64') + ':' + os.environ.get('LD_LIBRARY_PATH', ''))
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600, env=env)
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith('case=')]
    assert len(lines) == 4, r.stdout + r.stderr
    if any('nvrtc' in ln.lower() and 'libnvrtc' in ln.lower() for ln in lines):
        pytest.skip('NVRTC not available: ' + r.stdout)
    assert r.returncode == 0, r.stdout + r.stderr
