"""bench.py's output contract, checked on the CPU: the reference arm (the FP64
oracle on a bounded sample of the workload) prints one JSON line with the
keys the driver reads, and the roofline arithmetic helpers count what the
path computes."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    res = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "1", "--workload", "small_2d_n5"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert d["warmup"] >= 3                                  # at least three warm-up steps


def test_algorithmic_operation_count():
    sys.path.insert(0, ROOT)
    import bench
    ops = bench.algorithmic_ops_per_pixel(32, 5, True)
    # N (n + 2) channel accumulations, twice with interpolation; n(n+1)/2 + n
    # Newton-Girard; 6 for CF and weighting
    assert ops == {"main": 448, "newton_girard": 20, "cf": 6, "beam_total": 474}
    assert bench.algorithmic_ops_per_pixel(256, 3, False)["beam_total"] == 256 * 5 + 9 + 6


def test_serving_and_ng_variants_are_named_keys_not_the_value():
    sys.path.insert(0, ROOT)
    import bench
    assert set(bench.NG_PREC) == {"cf32", "f64", "f32"}
    assert "compensated" in bench.NG_TEXT["cf32"]
