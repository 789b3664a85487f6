"""Host-side pieces of bench.py that need no GPU: the reference arm's JSON
line (the oracle timed on the host cores) and the stored series energies."""
import argparse
import io
import json
import os
import subprocess
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_line_keys(monkeypatch):
    calls = []

    def fake_rate(target_s=10.0, max_rows=None, threads=None):
        calls.append(target_s)
        return 1.5e8, 16, "100 of 80358 operator rows", 0.25

    monkeypatch.setattr(bench, "cpu_oracle_rate", fake_rate)
    args = argparse.Namespace(steps=2, warmup=3, gpus=1)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    assert len(calls) == 5
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "interactions/s" and line["higher_is_better"] is True
    assert line["steps"] == 2 and line["warmup"] == 3 and line["n_gpus"] == 1
    assert line["value"] == 1.5e8 and abs(line["ms_per_step"] - 250.0) < 1e-9
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 16
    assert line["e2e"] == {"value": 1.5e8, "unit": "interactions/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"] == "kirkwood_sphere"
    # the same config dict as the GPU arm states it (workload keys, N, parallelism, cache note)
    assert line["config"] == bench.kirkwood_config(80358, 1)


def test_reference_arm_loads_no_cuda_library():
    """The oracle arm runs in a process that never maps the CUDA library."""
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "bench.cpu_oracle_rate = lambda **k: (1.0e8, 1, 'stub', 0.01); "
            "sys.argv = ['bench.py', '--impl', 'reference', '--steps', '1', '--warmup', '3']; bench.main(); "
            "maps = open('/proc/self/maps').read(); "
            "assert '/libibim.so' not in maps, 'libibim.so mapped'; print('maps-ok')" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    assert "maps-ok" in r.stdout
    line = json.loads([ln for ln in r.stdout.splitlines() if ln.startswith("{")][-1])
    assert line["impl"] == "reference" and line["config"]["N"] > 70000


def test_oracle_rate_on_a_short_sample():
    import oracle
    v, cores, desc, dt = bench.cpu_oracle_rate(target_s=0.3)
    assert v > 0 and cores >= 1 and dt > 0 and "operator rows" in desc
    all_threads = oracle.num_threads()
    v1, c1, desc1, dt1 = bench.cpu_oracle_rate(target_s=0.3, threads=1)
    assert v1 > 0 and c1 == 1 and dt1 > 0
    assert oracle.num_threads() == all_threads  # restored after the single-core sample


def test_series_energies_by_workload():
    g = bench._series_kcal(bench.WORKLOAD)
    assert g is not None and -410.0 < g < -400.0
    assert bench._series_kcal(bench.TREECODE) is not None
    assert bench._series_kcal(dict(bench.WORKLOAD, kappa=0.2)) is None
