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
