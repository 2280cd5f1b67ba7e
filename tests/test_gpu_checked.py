"""The bounds-checked build (EG_CHECKED) on a sweep of small shapes, extents
1..5 in 1D-5D: results equal the oracle's, and no kernel computed an index
outside its arrays (a miss would make the call fail with EG_ERR_INTERNAL).
The sweep runs in a child process so that it loads libeg_checked.so alone."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_small_shape_sweep():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    env = dict(os.environ, EG_CHECKED_LIBRARY="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_sweep.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1].startswith("OK ")
