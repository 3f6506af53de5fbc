import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running statistical check")


def golden_path(name):
    return os.path.join(ROOT, "tests", "golden", name)


def paper_value(name):
    with open(golden_path("paper_values.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            parts = line.split()
            if parts[0] == name:
                return float(parts[1]), int(parts[2])
    raise KeyError(name)


@pytest.fixture(scope="session")
def gpu_lib():
    """Builds (if stale) and loads the CUDA library; GPU tests only."""
    from paper_2601_23252_gb300 import build, native
    build.build()
    return native.lib()
