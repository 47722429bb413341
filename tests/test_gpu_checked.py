"""The bounds-checked library (the same sources compiled with FSLBM_CHECKED:
every cell index a kernel reads from a segment record or a cell list, every
source cell a fast path forms by offset arithmetic, and the interior
precondition of the interface kernels are tested before the access) passes
the whole GPU suite: no check fires on any of its cases (a fired check makes
the next synchronising call raise), and every parity bar holds as it stands.
The suite runs in a child process with FSLBM_CHECKED=1, where the session
fixture of conftest.py asserts that the checked library is the one loaded."""
import os
import subprocess
import sys

import pytest

from paper_1409_5645_gb300 import build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(os.environ.get("FSLBM_CHECKED") == "1", reason="this is the run under the checked library")
def test_gpu_suite_under_the_checked_library():
    build.build(checked=True)
    env = dict(os.environ, FSLBM_CHECKED="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "tests", "-m", "gpu", "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=3600)
    tail = r.stdout[-4000:] + r.stderr[-2000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail
