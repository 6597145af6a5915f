import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


@pytest.fixture(autouse=True)
def _bounds_checked(request):
    """Under NIF_BOUNDS_BUILD=1 (the bounds-checked library, see
    tests/test_gpu_bounds.py) every GPU test must end with no failed index
    check."""
    yield
    if os.environ.get("NIF_BOUNDS_BUILD") != "1" or request.node.get_closest_marker("gpu") is None:
        return
    from paper_2604_24666_gb300 import nif
    enabled, failures = nif.nif_bounds_check()
    assert enabled, "NIF_BOUNDS_BUILD=1 but the loaded library is not the bounds build"
    assert failures == 0, f"{failures} failed index checks"
