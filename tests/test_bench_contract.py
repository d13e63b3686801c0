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


def _fake_sections():
    """Side sections shaped like the bench's own (every key the headline reads, long strings included)."""
    tc = lambda v, f, e: {"value": v, "roofline": {"frac": f, "kernel": "k" * 60}, "check": {"rel_l2": e},
                          "ms_per_step": 1.234567, "launches": 12345}
    by_block = {str(b): {"blocks": 123456, "deadline_ms": b / 48.0, "p50_ms": 0.1234567, "p99_ms": 0.98765432,
                         "miss_frac": 0.0123456} for b in (32, 64, 128, 256)}
    return {
        "shared_ir": {"workload": "w" * 200, "bf16split": tc(1.9e14, 0.71, 4.7e-6), "bf16": tc(4.8e14, 0.63, 1.7e-3),
                      "fp32": tc(2.3e13, 0.57, 2.9e-7), "cpu_baseline": {"sample": "s" * 300}},
        "mimo": {"bf16split": tc(2.3e14, 0.84, 5.2e-6), "bf16": tc(5.6e14, 0.71, 2.5e-3), "fp32": tc(2.7e13, 0.67, 3e-7)},
        "mono": {"p99_ms": 0.05123456, "deadline_ms": 1.3333333, "one_shot_ms": 0.5123456,
                 "offline": {"long_signal_1s_ir": {"tensor_bf16split": {"frac_of_bf16_peak": 0.7731234},
                                                   "tensor_bf16": {"frac_of_bf16_peak": 0.4581234}}}},
        "q15": {"dp2a": {"tap_macs_per_s": 1.81e13}, "roofline": {"frac": 0.9006}, "forms_agree_bitwise": True,
                "e2e": {"value": 1.79e13}},
        "ext": {"zero_gating": {"speedup": 1.4322, "bit_identical": True}, "crossfade": {"overhead": 0.1869}},
        "serving": {"capacity": {"batched": {"streams": 3200}, "per_stream": {"streams": 26},
                                 "per_stream_async": {"streams": 51}},
                    "groups": {"bf16split": {"channels": 18432}, "fp32": {"channels": 5120}},
                    "trace": {"seconds": 60.0, "max_active": 1400, "p50_ms": 0.1412345, "by_block": by_block}},
        "latency": {"p99_ms": 0.31234567, "deadline_ms": 2.6666667},
        "autotune_push_ms_per_sample": {"1024": 8.5e-05, "8192": 6.8e-05},
    }


def test_headline_is_compact_and_complete():
    """The headline (the bench's last line) keeps the contract's keys and fits the tail the driver reads."""
    line = {"impl": "ours", "metric": bench.METRIC, "value": 2.38e13, "unit": "tap-MAC/s", "n_gpus": 1, "steps": 20,
            "warmup": 5, "ms_per_step": 61.91234567, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic", "config": bench.workload_config(8192),
            "roofline": {"bound": "alu", "achieved": 48.51234, "peak": 80.5, "unit": "TFLOP/s", "frac": 0.6031234,
                         "traffic": 35700000.0, "kernel": "k1_gather (FP32 FMA gather)", "peak_basis": "p" * 80,
                         "k1_launches": 1234, "k1_avg_ms": 0.0512345, "k1_share_of_step": 0.95123,
                         "frac_at_measured_clock": 0.6031234},
            "cpu_baseline": {"value": 2.4e10, "unit": "tap-MAC/s", "cores": 16, "kind": "oracle", "sample": "s" * 200,
                             "cpu_seconds": 1.0, "samples_per_s": 5e5, "realtime_factor_per_core": 0.88,
                             "cpu_model": "Neoverse-V2"},
            "e2e": {"value": 2.2e13, "unit": "tap-MAC/s", "h2d_bytes_per_step": 368640000,
                    "d2h_bytes_per_step": 135167744, "ms_per_step": 66.1234, "path": "p" * 120},
            "clocks": {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "sm_min_mhz": 1920.0, "reasons": ["sw_power_cap"],
                       "samples": 10},
            "gpu_launches": 12345, "check": {"sampled_outputs": 64, "rel_l2": 2.8e-7, "max_abs": 1.2e-8,
                                             "against": "Eq. (4) at each output, float64"},
            "realtime_streams_48k": 9912.3456}
    h = bench.headline(line, _fake_sections())
    text = json.dumps(h)
    assert len(text) <= bench.HEADLINE_MAX, len(text)
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks",
              "gpu_launches"):
        assert k in h, k
    assert h["impl"] == "ours" and h["config"]["workload"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in h["roofline"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in h["e2e"], k
    # With sections of this size every side summary still fits.
    assert {"shared_ir", "mimo", "serving", "q15"} <= set(h["side"]), h["side"].keys()
    assert h["side"]["serving"]["trace"]["p99_ms"]["32"] > 0
