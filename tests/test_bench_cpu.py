"""bench.py's reference arm (the FP64 oracle on the host cores) prints one JSON
line with the keys of the bench contract; runs without a GPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    res = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--ref-inner", "2"],
                         capture_output=True, text=True, cwd=ROOT, timeout=600)
    assert res.returncode == 0, res.stderr[-2000:]
    lines = [l for l in res.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, res.stdout
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["dtype"] == "f64" and d["value"] > 0
    assert d["config"]["nr"] == 512 and d["config"]["nz"] == 4096
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the reference arm names the GPU arm's workload and default launch shape
    sys.path.insert(0, ROOT)
    import bench
    from paper_1408_5853_gb300 import ccell, inputs
    cfg = inputs.production_case()
    assert d["config"] == bench.headline_config(cfg, 1000, 1, bench.DEFAULT_FP64_LAUNCH)
    sol = ccell.Solver(inputs.small_case(q0=1.0))
    try:
        assert ccell.cc_get_launch(sol.ctx) == bench.DEFAULT_FP64_LAUNCH
    finally:
        sol.close()
