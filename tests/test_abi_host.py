"""The C-ABI library builds, loads without a GPU, exports every entry point
declared in include/smc.h, and its host-side utilities (normal quantile,
Eq. 4, Eq. 5) agree with the oracle and with SciPy."""
import ctypes
import os
import re
import subprocess
import sys

import numpy as np
import pytest
from scipy import special

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope='module')
def native():
    from paper_0912_2551_gb300 import _native
    _native.load()
    return _native


def _declared():
    txt = open(os.path.join(ROOT, 'include', 'smc.h')).read()
    txt = re.sub(r'/\*.*?\*/', '', txt, flags=re.S)
    return sorted(set(re.findall(r'\b(smc_[a-z_0-9]+)\s*\(', txt)))


def test_every_declared_symbol_is_exported(native):
    lib = native.LIB_PATH
    out = subprocess.run(['nm', '-D', '--defined-only', lib], capture_output=True, text=True).stdout
    exported = set(re.findall(r' T (smc_[a-z_0-9]+)', out))
    declared = _declared()
    assert declared, 'no declarations parsed'
    missing = [d for d in declared if d not in exported]
    assert not missing, missing
    for d in declared:
        assert d in native.SIGNATURES, f'{d} has no binding'


def test_create_without_gpu_reports_no_device(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip('a GPU is present')
    h = ctypes.c_void_p()
    assert native.smc_create(ctypes.byref(h), 0) == native.SMC_E_NO_DEVICE
    assert native.smc_strerror(native.SMC_E_NO_DEVICE) == b'no suitable CUDA device'


def test_as241_against_scipy(native):
    for p in [1e-12, 1e-6, 0.01, 0.025, 0.3, 0.5, 0.7, 0.975, 0.995, 0.99995, 1 - 1e-9]:
        z = native.smc_normal_quantile(p)
        assert abs(z - special.ndtri(p)) <= 4e-15 * max(1.0, abs(z)), p


def test_wilson_host_matches_oracle(native, orc):
    from oracle import wilson
    import paper_0912_2551_gb300 as smc
    for yes, n in [(0, 10), (10, 10), (253, 2648), (19, 2648), (1547, 2495), (7, 1000000)]:
        for conf in (0.95, 0.99, 0.9999):
            lo, hi = smc.wilson_interval(yes, n, conf)
            _, olo, ohi = wilson.wilson_interval(yes, n, conf)
            assert abs(lo - olo) <= 1e-12 * max(abs(olo), 1e-300) + 1e-300
            assert abs(hi - ohi) <= 1e-12 * abs(ohi)
    for p in [0.0, 0.01, 0.5, 0.9, 1.0]:
        a = smc.wilson_sample(p, 0.025, 0.99)
        b = wilson.wilson_sample_real(p, 0.025, 0.99)
        assert abs(a - b) <= 1e-9 * b


def test_formula_postfix():
    import paper_0912_2551_gb300 as smc
    f = ('U', 0.0, 200.0, ('atom', 0), ('and', ('atom', 1), ('F', 0.0, 50.0, ('atom', 2))))
    nodes = smc.postfix(f)
    assert [n[0] for n in nodes] == [2, 2, 2, 8, 4, 7]
    assert nodes[3][2:] == (0.0, 50.0) and nodes[5][2:] == (0.0, 200.0)


def test_missing_library_fails_loudly(tmp_path):
    """No fallback: with the library absent (and no rebuild), the binding
    raises instead of computing anything on the CPU; and no module of the
    package imports the oracle."""
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "from paper_0912_2551_gb300 import _native\n"
        "_native.LIB_PATH = %r\n"
        "_native._lib = None\n"
        "try:\n"
        "    _native.load(build_if_missing=False)\n"
        "except RuntimeError as e:\n"
        "    print('raised:', e)\n"
        "else:\n"
        "    print('loaded')\n" % (ROOT, str(tmp_path / 'missing' / 'libsmc.so')))
    r = subprocess.run([sys.executable, '-c', code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith('raised:'), r.stdout
    pkg = os.path.join(ROOT, 'paper_0912_2551_gb300')
    for name in os.listdir(pkg):
        if name.endswith('.py'):
            src = open(os.path.join(pkg, name)).read()
            assert not re.search(r'^\s*(from|import)\s+oracle\b', src, flags=re.M), name


def test_fig2_step_matches_oracle_procedure(native, orc):
    """smc_fig2_next_batch, driven over Bernoulli verdict streams, gives the
    batch sequence and totals of the oracle's Fig. 2 (oracle/wilson.py), for
    the iterative, conservative and fixed-size modes."""
    from oracle import wilson
    rng = np.random.default_rng(7)
    for p_true in (0.0, 0.003, 0.1, 0.5, 0.93, 1.0):
        for eps, conf in ((0.025, 0.99), (0.01, 0.95), (0.002, 0.95)):
            stream = rng.random(400000) < p_true

            def run(begin, count):
                return int(stream[begin:begin + count].sum()), count

            ref = wilson.iterative(run, eps, conf)
            sizes, n_tot, yes = [], 0, 0
            nxt = ctypes.c_uint64()
            while True:
                assert native.smc_fig2_next_batch(native.SMC_ITERATIVE, 0, conf, eps, yes, n_tot, n_tot,
                                                  ctypes.byref(nxt)) == 0
                if nxt.value == 0:
                    break
                y, _ = run(n_tot, nxt.value)
                sizes.append(nxt.value)
                yes += y
                n_tot += nxt.value
            assert sizes == ref['sizes'] and n_tot == ref['n_tot'] and yes == ref['yes'], (p_true, eps, conf)
            assert native.smc_fig2_next_batch(native.SMC_CONSERVATIVE, 0, conf, eps, 0, 0, 0, ctypes.byref(nxt)) == 0
            assert nxt.value == wilson.wilson_sample(0.5, eps, conf)
            assert native.smc_fig2_next_batch(native.SMC_CONSERVATIVE, 0, conf, eps, 3, 10, 10,
                                              ctypes.byref(nxt)) == 0 and nxt.value == 0
    assert native.smc_fig2_next_batch(native.SMC_FIXED_N, 777, 0.95, 0.0, 0, 0, 0, ctypes.byref(nxt)) == 0
    assert nxt.value == 777
    assert native.smc_fig2_next_batch(native.SMC_FIXED_N, 777, 0.95, 0.0, 5, 777, 777, ctypes.byref(nxt)) == 0
    assert nxt.value == 0
    # Table 1 / Fig. 2: the first iterative batch at 99%, eps = 0.025 is 127
    assert native.smc_fig2_next_batch(native.SMC_ITERATIVE, 0, 0.99, 0.025, 0, 0, 0, ctypes.byref(nxt)) == 0
    assert nxt.value == 127
    bad = [(99, 0, 0.95, 0.01, 0, 0, 0), (native.SMC_ITERATIVE, 0, 1.0, 0.01, 0, 0, 0),
           (native.SMC_ITERATIVE, 0, 0.95, 0.5, 0, 0, 0), (native.SMC_ITERATIVE, 0, 0.95, 0.01, 5, 4, 10),
           (native.SMC_ITERATIVE, 0, 0.95, 0.01, 1, 11, 10), (native.SMC_FIXED_N, 0, 0.95, 0.01, 0, 0, 0)]
    for args in bad:
        assert native.smc_fig2_next_batch(*args, ctypes.byref(nxt)) == native.SMC_E_INVALID_ARG, args
    assert native.smc_fig2_next_batch(native.SMC_ITERATIVE, 0, 0.95, 0.01, 0, 0, 0, None) == \
        native.SMC_E_INVALID_ARG
