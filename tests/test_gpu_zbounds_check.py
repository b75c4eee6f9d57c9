"""The bounds-checking build: the library compiled with -DLU_BOUNDS_CHECK,
whose index guards (pivot rows of the panels, solve block tickets) record a
status bit and take a safe path instead of an out-of-range access, runs the
panel, solve and batched tests in a child process; no guard may fire (a fired
guard surfaces as LU_EINTERNAL from the status reads those tests make)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bounds_checking_build_runs_clean():
    from paper_2202_13995_gb300 import build
    lib = build.build(bounds_check=True)
    env = dict(os.environ, GB300LU_LIB=lib)
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
           "-k", "panel or factor_solve or multi_rhs or mixed_refine or batched",
           "tests/test_gpu_steps.py", "tests/test_gpu_solve.py", "tests/test_gpu_batched.py"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
