import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
HERE = os.path.dirname(os.path.abspath(__file__))
if HERE not in sys.path:
    sys.path.insert(0, HERE)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (run with -m gpu)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


_MEASURED = []


@pytest.fixture
def report(request):
    """Records a measured figure of the test (an error against the oracle, a
    convergence sequence): printed with the test and repeated in the
    terminal summary, so a quiet run (-q) still shows it."""
    def _report(line: str) -> None:
        text = f"{request.node.name}: {line}"
        print(text)
        _MEASURED.append(text)
    return _report


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if _MEASURED:
        terminalreporter.section("measured figures")
        for line in _MEASURED:
            terminalreporter.write_line(line)
