"""Host-side checks of bench.py on the CPU: the reference arm's JSON line (it times the oracle on the host
cores) carries the contract's keys, and the bench's float64 self-check form of Eq. 4 agrees with the oracle.
"""
import json
import os
import subprocess
import sys

import numpy as np

import bench
import oracle
from paper_2401_01607_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0",
                        "--ref-samples", "300"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["config"]["workload"] and line["scaling"] == "weak"
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert cb["samples_per_s"] > 0 and cb["realtime_factor_per_core"] > 0
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_bench_self_check_form_of_eq4_matches_the_oracle():
    rng = np.random.default_rng(4)
    x = synth.audio(3000, 41)
    H = np.stack([synth.decayed_ir(700, 140.0, 42 + v) for v in range(3)])
    vstart = np.array([0, 1000, 1001], np.int64)
    for m in [0, 1, 699, 700, 1000, 1001, 1500, 2999, 3000, 3698] + list(rng.integers(0, 3699, 20)):
        a = bench.eq4_at(x, H, vstart, int(m))
        b = oracle.direct_at(x, H, vstart, int(m))
        assert abs(a - b) <= 1e-12 * max(1.0, abs(b)), (m, a, b)
