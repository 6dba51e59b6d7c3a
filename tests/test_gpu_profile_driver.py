"""The profiling driver behind profiles/: a state saved after equilibration (bench.py --profile
--save-state) is loaded by a later profiled run (--load-state) of the same system."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], capture_output=True, text=True,
                       cwd=ROOT, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("extra", [[], ["--cg-mode", "1"]])
def test_saved_state_feeds_the_profiled_run(tmp_path, extra):
    path = str(tmp_path / "eq.npz")
    saved = run("--profile", "1", "--molecules", "3000", "--save-state", path, "--equilibrate", "200")
    assert saved["steps"] == 200 and os.path.exists(path)
    d = np.load(path)
    assert d["x"].shape == (12000, 3) and d["v"].shape == (12000, 3) and np.isfinite(d["x"]).all()
    prof = run("--profile", "10", "--molecules", "3000", "--load-state", path, *extra)
    assert prof["profile_steps"] == 10 and prof["atoms"] == 12000
    assert prof["lists"]["n_hr"] > 0 and prof["lists"]["n_cg"] > 0
