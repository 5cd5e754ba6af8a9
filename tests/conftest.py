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
    from tests.helpers import PARITY, REPORT
    if REPORT:
        terminalreporter.write_sep("-", "largest parity errors seen")
        for k in sorted(REPORT):
            terminalreporter.write_line(f"{k}: {REPORT[k]:.3e}")
    if PARITY:
        terminalreporter.write_sep("-", "parity coverage (pixels / elements checked, branch outcomes)")
        for k in sorted(PARITY):
            c = PARITY[k]
            if "pixels" in c:
                px = max(c["pixels"], 1)
                terminalreporter.write_line(
                    f"{k}: {c['pixels']} pixels, unchecked {c['excluded']} ({c['excluded'] / px:.2e}), "
                    f"with several admissible outcomes {c['branched']} ({c['branched'] / px:.2e}), "
                    f"matched only a non-FP64 outcome {c['other_branch']} ({c['other_branch'] / px:.2e})")
            else:
                terminalreporter.write_line(f"{k}: " + ", ".join(f"{a} {b}" for a, b in c.items()))
