import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    """Parse a tests/golden/*.txt fixture: '[section]' headers and 'key: value' lines, '#' comments."""
    path = os.path.join(ROOT, "tests", "golden", name)
    out, cur = {}, None
    for raw in open(path):
        line = raw.split("#", 1)[0].strip()
        if not line:
            continue
        if line.startswith("[") and line.endswith("]"):
            cur = out.setdefault(line[1:-1], {})
            continue
        k, v = (t.strip() for t in line.split(":", 1))
        (cur if cur is not None else out)[k] = v
    return out


@pytest.fixture(scope="session")
def golden():
    return load_golden
