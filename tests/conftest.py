import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter):
    from tests.helpers import REPORT
    if REPORT:
        terminalreporter.write_sep("-", "largest parity errors seen")
        for k in sorted(REPORT):
            terminalreporter.write_line(f"{k}: {REPORT[k]:.3e}")
