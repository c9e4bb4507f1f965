"""Host-side helpers of the bench and the corrector (no GPU)."""
import os

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_kernel_hash_and_recorded_traffic_lookup():
    import bench
    h = bench.kernel_source_hash()
    assert len(h) == 12
    lines = [l.split() for l in open(os.path.join(ROOT, "profiles", "ncu_traffic.txt")) if not l.startswith("#")]
    assert lines and all(len(l) == 4 and int(l[2]) > 0 for l in lines)
    # a lookup returns the bytes only for the recorded kernel, size and source hash
    rec = {(l[0], l[1]): (int(l[2]), l[3]) for l in lines}
    b, src = rec[("rhs_E", "256")]
    assert bench.ncu_traffic("rhs_E", 256) == (float(b) if src == h else None)
    assert bench.ncu_traffic("rhs_E", 128) is None
    assert bench.ncu_traffic("line_x_mass", 256) is None


def test_corrector_weights_roundtrip(tmp_path):
    from paper_2103_06998_gb300 import adi, corrector, inputs
    flat = adi.net_flatten(inputs.net_init(3))
    path = str(tmp_path / "w.f32")
    corrector.save(flat, path)
    np.testing.assert_array_equal(corrector.load(path), flat)
    # the committed weights have the documented size and are finite
    w = corrector.load()
    assert w.size == adi.NET_PARAMS and np.all(np.isfinite(w))
    # their padding entries are zero (layer 0 ci >= 9, layer 3 co >= 6)
    real = adi.net_flatten([(np.ones((3, 3, 3, ci, co)), np.ones(co)) for ci, co in adi.NET_REAL]) != 0
    assert np.all(w[~real] == 0.0)


def test_reference_arm_prints_the_contract_line():
    # the oracle arm of bench.py on a small case: one JSON line with the keys
    # of the main arm's line, the same config keys, and its own e2e/cpu_baseline
    import json
    import subprocess
    import sys
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "12",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert set(d["config"]) == {"workload", "n", "p", "tau", "l2", "parallelism"} and d["config"]["n"] == 12
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert "fits in the 129 MB L2" in d["config"]["l2"]


def test_clock_summary_parses_samples_and_throttle_reasons():
    # the bench's clock record from nvidia-smi CSV rows (no GPU: rows written by hand)
    import bench
    c = bench.ClockSampler(0)
    rows = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
            "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
            "0, 2040, 2070, 1200.5, 0x0, Not Active, Not Active, Not Active, Not Active",
            "garbage line", "0, [N/A], 2070, 1, 0x0, a, b, c, d"]
    c.f.write("\n".join(rows) + "\n")
    s = c.summary()
    assert s["samples"] == 3 and s["sm_mhz"] == 2040 and s["sm_max_mhz"] == 2070
    assert s["reasons"] == ["sw_power_cap"]
    c2 = bench.ClockSampler(0)
    c2.f.write("0, 1500, 2070, 1400, 0x8, Active, Not Active, Active, Not Active\n")
    assert c2.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    c3 = bench.ClockSampler(0)
    assert c3.summary()["reasons"] == ["nvidia-smi unavailable"]
