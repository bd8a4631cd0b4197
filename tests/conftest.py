import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))
for p in (ROOT, HERE):
    if p not in sys.path:
        sys.path.insert(0, p)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """The achieved errors of every unwrap compared with the FP64 oracle in this run."""
    import parity_log
    lines = parity_log.table()
    if lines:
        terminalreporter.section("achieved errors against the FP64 oracle")
        for ln in lines:
            terminalreporter.write_line(ln)
