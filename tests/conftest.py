import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


@pytest.fixture(scope="session")
def oracle_lib():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Prints the parity comparisons against the plain bars (no FP32
    conditioning allowances) that the GPU tests recorded."""
    gu = sys.modules.get("gpu_util")
    lines = getattr(gu, "REPORT", None) if gu else None
    if lines:
        terminalreporter.section("parity against the plain bars")
        for ln in lines:
            terminalreporter.write_line(ln)
