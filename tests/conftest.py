import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds on CPU")


@pytest.fixture(scope="session")
def paper_values():
    with open(os.path.join(GOLDEN, "paper_values.json")) as f:
        return json.load(f)


@pytest.fixture(autouse=True)
def _checked_build_is_clean(request):
    """With FFA_LIBRARY=checked (the bounds-checked library), every GPU test must leave
    no recorded index violation."""
    yield
    if os.environ.get("FFA_LIBRARY") != "checked" or request.node.get_closest_marker("gpu") is None:
        return
    import paper_2004_03701_gb300 as ffa
    checked, bits = ffa.checked_status()
    assert checked, "FFA_LIBRARY=checked but the loaded library is not the checked build"
    assert bits == 0, "the checked build recorded an index out of range (bits 0x%x)" % bits
