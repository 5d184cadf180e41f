import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.dirname(os.path.abspath(__file__))
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Print (and optionally write) the element-wise parity report of the GPU tests."""
    try:
        from parity_metrics import REPORT
    except ImportError:
        return
    if not REPORT["elementwise"] and not REPORT["log_alpha"]:
        return
    import json
    text = json.dumps(REPORT, indent=1, sort_keys=True)
    terminalreporter.write_sep("-", "element-wise parity report (worst error / (|oracle| + posterior sd))")
    terminalreporter.write_line(text)
    path = os.environ.get("AUX_PARITY_REPORT")
    if path:
        with open(path, "w") as f:
            f.write(text + "\n")
