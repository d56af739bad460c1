import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (runs the sm_103a library)")
    config.addinivalue_line("markers", "slow: larger CPU cases")


def read_golden(name):
    """Parse a tests/golden fixture: keyword lines and numeric table rows."""
    path = os.path.join(ROOT, "tests", "golden", name)
    kv, rows = {}, []
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            parts = line.split()
            try:
                rows.append([float(p) for p in parts])
            except ValueError:
                kv[parts[0]] = [float(p) for p in parts[1:]]
    return kv, rows
