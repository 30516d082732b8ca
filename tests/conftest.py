import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the CUDA library)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library (fails loudly if it was not built)."""
    from paper_2407_17296_gb300 import binding
    return binding.load()


def pytest_sessionfinish(session, exitstatus):
    """Write the near-tie counts of the GPU parity tests that ran (tests/parity.py TIE_REPORT)
    as JSON to the file $SMC2_TIE_REPORT names (nothing is written when it is unset)."""
    import json
    try:
        from tests.parity import TIE_REPORT
    except ImportError:
        return
    path = os.environ.get("SMC2_TIE_REPORT")
    if not TIE_REPORT or not path:
        return
    with open(path, "w") as f:
        json.dump(TIE_REPORT, f, indent=1, sort_keys=True)
