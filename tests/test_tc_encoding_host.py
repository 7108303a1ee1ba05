"""The tcgen05 encodings of the surrogate's inference kernel
(paper_0912_2551_gb300/csrc/smc_tc.h), compiled for the host and checked by
tests/tc_encoding_check.cpp: the K-major core-matrix operand layout is a
bijection with the strides the kernel's descriptors state, and the
shared-memory and instruction descriptors carry each field at the bit
positions the PTX ISA documents."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tc_encodings(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None:
        pytest.skip('no g++')
    exe = str(tmp_path / 'tc_encoding_check')
    subprocess.run([gxx, '-O1', '-std=c++17', '-I', os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc'),
                    os.path.join(ROOT, 'tests', 'tc_encoding_check.cpp'), '-o', exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith('ok'), r.stdout + r.stderr
