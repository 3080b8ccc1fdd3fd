import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: CPU test that takes more than a few seconds")


def load_golden_sections(name):
    """Parse a golden text fixture into {section title: ndarray}."""
    out = {}
    cur = None
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line.startswith("# section:"):
                if cur is not None:
                    out[cur] = np.array(rows, dtype=np.float64)
                cur = line[len("# section:"):].strip().split(" ")[0]
                rows = []
            elif line and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    if cur is not None:
        out[cur] = np.array(rows, dtype=np.float64)
    return out


@pytest.fixture
def golden():
    return load_golden_sections
