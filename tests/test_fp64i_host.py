"""The integer-pipe binary64 division and logarithm of the FP64 SSA path
(paper_0912_2551_gb300/csrc/smc_fp64i.h), compiled for the host and checked
against the platform's arithmetic by tests/fp64i_check.cpp: the division
bit for bit against IEEE-754 division on 10^6 operand pairs of every class,
the logarithm within 0.502 ulp of long-double logl and correctly rounded on
more than 99.99% of 1.75 x 10^6 arguments (the SSA's uniforms, values near
1, the table's bucket edges, general positive doubles), and the SSA's form
-ln((2v + 1) 2^-53) from the integer equal bit for bit to -ln u; the exact
integer-pipe conversion of integers bit for bit against the IEEE
conversion; and the step of Eq. 2a as the event loop forms it,
tau = -ln u / a_0 rounded once from the fixed-point logarithm and a 64-bit
reciprocal, within 0.51 ulp of the long-double quotient."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fp64i_against_host_arithmetic(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None:
        pytest.skip('no g++')
    if np.finfo(np.longdouble).nmant < 60:
        pytest.skip('no extended-precision long double on this platform')
    exe = str(tmp_path / 'fp64i_check')
    subprocess.run([gxx, '-O2', '-std=c++17', '-I', os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc'),
                    os.path.join(ROOT, 'tests', 'fp64i_check.cpp'), '-o', exe, '-lm'], check=True)
    r = subprocess.run([exe, '1000000'], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    kv = dict(f.split('=', 1) for f in r.stdout.strip().splitlines()[-1].split())
    assert int(kv['div_mismatches']) == 0
    assert float(kv['log_max_ulp']) <= 0.502
    assert float(kv['log_correctly_rounded']) >= 0.9999
    assert int(kv['neglog53_mismatches']) == 0
    assert int(kv['i2d_mismatches']) == 0
    # tau = -ln u / a_0 rounded once from the fixed-point logarithm and
    # reciprocal (relative error below 2^-60 before the rounding): within
    # 0.51 ulp, correctly rounded but for quotients within 2^-7 ulp of a midpoint
    assert float(kv['tau_max_ulp']) <= 0.51 and int(kv['tau_bad']) == 0
    assert float(kv['tau_correctly_rounded']) >= 0.99
