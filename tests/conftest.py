import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_terminal_summary(terminalreporter):
    """The achieved parity figures (tests.helpers.record), one JSON line per
    record, after the results: quiet runs print them too."""
    import json
    from tests.helpers import RECORDS
    if RECORDS:
        terminalreporter.section("parity figures")
        for r in RECORDS:
            terminalreporter.write_line(json.dumps(r, default=str))
