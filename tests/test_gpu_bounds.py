"""The index-checked build (libpflbm_bounds.so, compiled with -DPFLBM_BOUNDS)
runs the small parity cases through every 2D step kernel and the batched
kernels without a single refused access, and with FP32 still within the
parity bar of the FP64 oracle. It runs in a child process: a process loads
one build of the library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_index_checked_build_refuses_no_access():
    from paper_2312_00369_gb300 import pflbm
    assert os.path.exists(pflbm.BOUNDS_LIB_PATH), "libpflbm_bounds.so missing (build())"
    env = dict(os.environ, PFLBM_LIBRARY=pflbm.BOUNDS_LIB_PATH)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "bounds_cases.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    print(out)
    assert out["violations"] == 0
    for name, errs in out["cases"].items():
        for key, err in errs.items():
            bar = 1e-5 if key.startswith("fp32") else 2e-2
            assert err <= bar, (name, key, err)
