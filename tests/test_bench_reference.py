"""The reference arm of bench.py (the FP64 oracle timed on the host) prints
one JSON line with the keys the measurement contract asks for, and names a
charge-exchange channel added with --cx-sigma in its workload; run on the small
32x32x64 workload so that it takes seconds. The option is refused for the
ensemble."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_its_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "1", "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert "32x32x64" in line["cpu_baseline"]["sample"]


def test_reference_arm_with_charge_exchange_names_it():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "c1",
                          "--steps", "1", "--warmup", "3", "--cx-sigma", "1e-17"], cwd=ROOT, capture_output=True,
                         text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert "charge exchange" in line["config"]["workload"] and line["value"] > 0


def test_charge_exchange_option_refused_for_the_ensemble():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "c4", "--cx-sigma", "1e-17"],
                         cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.returncode != 0 and "--cx-sigma applies to c1-c3" in out.stderr
