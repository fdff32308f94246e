import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running")


@pytest.fixture
def save_report():
    """Writes a test's measured figures as JSON to $FDTD_RESULTS_DIR
    (default: results/ at the repository root)."""
    def save(name, obj):
        d = os.environ.get("FDTD_RESULTS_DIR") or os.path.join(ROOT, "results")
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name), "w") as f:
            json.dump(obj, f)
    return save
