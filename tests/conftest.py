import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103) and runs the CUDA library")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


@pytest.fixture(scope="session")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def pytest_terminal_summary(terminalreporter):
    """The parity bars measured on the oracle during the run (tests/oracle_bars.py), one line each."""
    mod = sys.modules.get("oracle_bars")
    if mod is None or not getattr(mod, "RECORD", None):
        return
    terminalreporter.section("parity bars measured on the oracle")
    for line in mod.RECORD:
        terminalreporter.write_line(line)
