import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(autouse=True, scope="session")
def _library_variant():
    """With FSLBM_CHECKED=1 the binding must have loaded the bounds-checked
    library (checked once, at the first test of the session)."""
    if os.environ.get("FSLBM_CHECKED") == "1":
        from paper_1409_5645_gb300 import fslbm
        assert fslbm.lib().fslbm_build_info() & 1, "FSLBM_CHECKED=1 but the normal library is loaded"
    yield
