import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Counts and measured errors that tests report (near-ties, flagged draws,
# quantisation errors): printed at the end of the run, passing or not.
REPORTS = []


def report(name, **values):
    """Record one line of measured values for the end-of-run summary."""
    REPORTS.append((name, values))


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    if not REPORTS:
        return
    terminalreporter.section("measured counts and errors")
    for name, values in REPORTS:
        terminalreporter.write_line(f"{name}: {json.dumps(values, sort_keys=True)}")
