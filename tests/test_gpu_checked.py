"""The checked build (-DMM_CHECKS: every guarded device access tests its index and
reports a failure as MM_EDEVICE) runs every shooting path without a failed check
and with the usual results. It runs in a child process, which loads the checked
library first."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_every_path_passes_its_bounds_checks():
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_run.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "without a failed bounds check" in r.stdout
