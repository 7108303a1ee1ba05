"""The trace monitor's window tests on the integer pipes (smc_nest.h): the
bounds nest_last_within / nest_first_reaching, compared on the CPU with
the rounded subtractions they replace, over window offsets and bounds of
every kind and times in the ulp neighbourhoods of the boundaries
(tests/nest_window_host.cpp)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_0912_2551_gb300', 'csrc')


def test_window_bounds_match_subtraction(tmp_path):
    gxx = shutil.which('g++')
    if gxx is None:
        pytest.skip('no g++')
    exe = str(tmp_path / 'nest_window_host')
    subprocess.run([gxx, '-O1', '-std=c++17', '-ffp-contract=off', '-I', CSRC, '-I', os.path.join(ROOT, 'include'),
                    os.path.join(ROOT, 'tests', 'nest_window_host.cpp'), '-o', exe], check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    cases, checks, bad, fb_ordinary, fb_extreme = (int(w) for w in r.stdout.split()[-5:])
    assert bad == 0
    assert checks > 100000 and cases > 100000
    # the subtraction fallback only near the top of the double range
    assert fb_ordinary == 0
