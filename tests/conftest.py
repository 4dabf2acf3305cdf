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
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    import parity_log
    reports = parity_log.report_lines()
    if reports:
        terminalreporter.write_sep("-", "error reports")
        for ln in reports:
            terminalreporter.write_line(ln)
    lines = parity_log.summary_lines()
    if lines:
        terminalreporter.write_sep("-", "parity exclusions (oracle-flagged borderline pixels / Gaussians)")
        for ln in lines:
            terminalreporter.write_line(ln)


@pytest.fixture(scope="session")
def orc():
    from oracle import oracle as O
    O.lib()
    return O
