"""The bounds-checked library (compiled with -DWSSR_CHECK_BOUNDS) and the
NaN-poisoned workspace (options.debug = WSSR_DEBUG_POISON), on the GPU paths
that keep state in the workspace between kernels: the history-averaged step,
checkpoint/resume, the randomized SVD and the plain tensor-core step with a
ragged parameter count (M % 64 != 0).

The checked build skips any out-of-range index or tensor map and reports
WSSR_ERR_BOUNDS; the poison makes every read of a workspace slot that no kernel
wrote produce NaN, which the steps report as WSSR_ERR_NONFINITE or which fails
the tests' parity checks. The selected test modules run unchanged in a child
process with both switched on (WSSR_CHECK_BOUNDS=1, WSSR_DEBUG_POISON=1).
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workspace_paths_under_bounds_checks_and_poison():
    from paper_2512_05749_gb300 import build
    build.build(checked=True)
    env = dict(os.environ, WSSR_CHECK_BOUNDS="1", WSSR_DEBUG_POISON="1")
    mods = ["tests/test_gpu_history.py", "tests/test_gpu_checkpoint.py", "tests/test_gpu_rssr.py"]
    sel = ["-k", "not matrix_free"]
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", *mods, *sel], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    assert p.returncode == 0, p.stdout[-4000:] + p.stderr[-2000:]
    p = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "tests/test_gpu_parity.py",
                        "-k", "test_step_bf16 and tcgen05 and 2040"], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert p.returncode == 0, p.stdout[-4000:] + p.stderr[-2000:]
    assert "passed" in p.stdout
