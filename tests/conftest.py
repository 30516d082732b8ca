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
    to $SMC2_TIE_REPORT, or to gpurun_out/parity_near_ties.json when that folder exists."""
    import json
    try:
        from tests.parity import TIE_REPORT
    except ImportError:
        return
    if not TIE_REPORT:
        return
    path = os.environ.get("SMC2_TIE_REPORT")
    if not path:
        out = os.path.join(ROOT, "gpurun_out")
        if not os.path.isdir(out):
            return
        path = os.path.join(out, "parity_near_ties.json")
    with open(path, "w") as f:
        json.dump(TIE_REPORT, f, indent=1, sort_keys=True)
