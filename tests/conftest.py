import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)
TESTS = os.path.join(ROOT, "tests")
if TESTS not in sys.path:
    sys.path.insert(0, TESTS)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")
    config.addinivalue_line("markers", "oracle16(*jobs): needs these N = 2^16 oracle jobs (tests/oracle_jobs.py)")


def read_golden(name):
    rows = {}
    lines = []
    with open(os.path.join(GOLDEN, name)) as f:
        for ln in f:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            lines.append(ln)
            parts = ln.split()
            rows[parts[0]] = parts[1:]
    return rows, lines


def pytest_collection_finish(session):
    """Start the N = 2^16 oracle jobs in spawned processes as soon as a test
    that needs them is selected, so they run while the other tests do."""
    names = set()
    for item in session.items:
        m = item.get_closest_marker("oracle16")
        if m is not None:
            names.update(m.args)
    if names:
        import oracle_jobs
        oracle_jobs.start(sorted(names))


def pytest_sessionfinish(session, exitstatus):
    mod = sys.modules.get("oracle_jobs")
    if mod is not None:
        mod.shutdown()
