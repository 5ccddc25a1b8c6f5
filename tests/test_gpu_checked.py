"""The checked build (libpic_gb300_checked.so, -DPIC_CHECKED): every cell,
slot and list index the particle kernels read from memory is tested before
use, and a bad one is reported (PIC_ESTATE, error bit ERR_BOUNDS) instead of
being followed. Runs of the tiny and small workloads in both stores, with
sorting, injection and ionization, must pass every check and keep the integer
moments of the FP64 oracle."""
import json
import os
import subprocess
import sys

import pytest

import oracle as O
from paper_2606_05893_gb300 import _build
from paper_2606_05893_gb300 import workloads as W
from tests.gpu_compare import compare_integer_moments

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
import paper_2606_05893_gb300 as pkg
from paper_2606_05893_gb300 import workloads as W
pkg.load_library()
out = {}
for name, wl, prec, steps in [("tiny64", W.config_tiny(seed=5), pkg.PIC_FP64, 10),
                              ("small64", W.config_small(seed=3, n_preload=3000), pkg.PIC_FP64, 6),
                              ("tinymx", W.config_tiny(seed=5), pkg.PIC_MIXED, 10)]:
    sim = pkg.Simulation(wl, precision=prec, cg_rtol=1e-13, cg_maxit=5000)
    sim.step(steps)
    out[name] = sim.moments()
    sim.close()
print(json.dumps(out))
"""


def test_checked_build_runs_clean_and_matches_oracle():
    lib = _build.build(checked=True)
    env = dict(os.environ, PIC_GB300_LIB=lib)
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    got = json.loads(r.stdout.strip().splitlines()[-1])
    for name, wl, steps in [("tiny64", W.config_tiny(seed=5), 10), ("small64", W.config_small(seed=3, n_preload=3000), 6)]:
        ref = O.Oracle(wl, cg_rtol=1e-13)
        ref.step(steps)
        compare_integer_moments(got[name], ref.moments())
        ref.close()
    assert got["tinymx"]["error_flags"] == 0
