"""The reference arm of bench.py (the FP64 oracle on the host cores) prints
one JSON line with the contract's keys, every number measured as it ran.
Runs on CPU only (no GPU needed): one whole 17^3 oracle load step, two at
one thread, and one pass each at 129^3."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, cwd=ROOT,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.strip().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "s/load-step" and d["higher_is_better"] is False
    for k in ("metric", "value", "n_gpus", "steps", "warmup", "ms_per_step", "scaling", "dtype",
              "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1
    assert len(cb["seconds"]) == 1 and cb["seconds"][0] > 0 and cb["cycles"][0] >= 1
    assert len(cb["one_thread"]["seconds"]) == 2
    for p in ("hessvec", "gradient", "energy_diff"):
        assert cb["passes_129"][p]["seconds"] > 0
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert max(d["config"]["pressure_steps"]) <= 5e-3
