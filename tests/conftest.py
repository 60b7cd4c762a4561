import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_ignore_collect(collection_path, config):
    """A GPU-only run (-m gpu) does not collect the CPU property tests when
    hypothesis, which their module needs at import, is not installed (the GPU
    box has no hypothesis): they would otherwise show up as a skipped module."""
    if collection_path.name != "test_oracle_properties.py" or config.getoption("markexpr") != "gpu":
        return None
    try:
        import hypothesis  # noqa: F401
    except ImportError:
        return True
    return None


@pytest.fixture(scope="session")
def golden_dir():
    return os.path.join(ROOT, "tests", "golden")
