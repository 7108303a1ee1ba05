"""bench.py on the CPU: the reference arm (the oracle timed on the host
cores, the only arm that runs without a GPU) prints one JSON line with the
keys of the benchmark contract, and the per-event operation counts behind
the issue roofline match a count by hand for Lotka-Volterra."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line(orc):
    r = subprocess.run([sys.executable, os.path.join(ROOT, 'bench.py'), '--impl', 'reference', '--steps', '1',
                        '--warmup', '3'], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip().startswith('{')]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d['impl'] == 'reference' and d['metric'] == bench.METRIC
    assert d['unit'] == 'trajectories/s' and d['value'] > 0 and d['higher_is_better'] is True
    assert d['steps'] == 1 and d['warmup'] == 3 and d['ms_per_step'] > 0
    assert d['scaling'] == 'weak' and d['vs_baseline'] is None and d['data'] == 'synthetic'
    assert 'workload' in d['config']
    cb = d['cpu_baseline']
    assert cb['kind'] == 'oracle' and cb['cores'] >= 1 and cb['value'] == d['value'] and cb['sample']
    e2e = d['e2e']
    assert e2e['value'] == d['value'] and e2e['unit'] == d['unit']
    assert e2e['h2d_bytes_per_step'] == 0 and e2e['d2h_bytes_per_step'] == 0


def test_ops_per_event_lotka_volterra():
    import bench
    import workloads
    model, _ = workloads.lotka_volterra()
    # Philox 40, two uniform maps 4, ln 1, clock 2, selection 2 x (R + 1) / 2
    # = 4, x += v_j: nnz of (+1), (-1, +1), (-1) = 4/3 on average, horizon 2,
    # atoms 2 x 2; propensities: FP64 path 3R = 9, mixed path 3 x mean
    # |dep(j)| = 3 x (2 + 3 + 2) / 3 = 7
    common = 40 + 4 + 1 + 2 + 4 + 4 / 3 + 2 + 4
    assert bench.algorithmic_ops_per_event(model, 2, True) == pytest.approx(common + 9)
    assert bench.algorithmic_ops_per_event(model, 2, False) == pytest.approx(common + 7)
