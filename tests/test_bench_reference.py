"""The reference arm of bench.py (the FP64 CPU oracle on the host cores) runs without a
GPU and prints one JSON line with the contract's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    # the sphere workload keeps this CPU test short; the default workload (the scale
    # case) runs the same code path with another mesh and stride
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3", "--workload", "sphere",
                        "--no-oracle-table"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["warmup"] >= 3 and d["higher_is_better"] is True
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["unit"] == "cell-velocity updates/s" and d["dtype"] == "f64"
    assert d["config"]["workload"].startswith("sphere") and d["config"]["K"] == 3033
    assert d["config"]["sample_K"] == len(range(0, 3033, 30))
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["h2d_bytes_per_step"] == 0


def test_default_workload_is_the_scale_case():
    """The bench line's workload is the largest single-GPU configuration: the
    ~500k-cell x ~8,000-velocity sphere-cone."""
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "bench.py")).read()
    assert 'ap.add_argument("--workload", default="scale"' in src
    assert bench.CPU_STRIDE["scale"] >= 1
