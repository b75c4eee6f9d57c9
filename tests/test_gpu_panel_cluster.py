"""The cluster panel kernel (FP32, one thread-block cluster, opt-in with
GB300LU_PANEL_CLUSTER): the panel and mixed-precision solve tests, run again
in a child process that selects it, must pass unchanged."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_panel_and_mixed_solves_with_the_cluster_panel():
    env = dict(os.environ, GB300LU_PANEL_CLUSTER="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-p", "no:cacheprovider",
           "tests/test_gpu_steps.py", "tests/test_gpu_solve.py", "tests/test_gpu_nopiv.py",
           "-k", "panel or mixed or nopiv"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout
