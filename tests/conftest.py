import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built CUDA library")


def read_table1():
    """Table 1 fixture: {(branch, q): (eps, [a0..aq])}."""
    rows = {}
    with open(os.path.join(GOLDEN, "table1_minimax.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows[(parts[0], int(parts[1]))] = (float(parts[2]), [float(v) for v in parts[3:]], parts[3:])
    return rows


@pytest.fixture(scope="session")
def table1():
    return read_table1()


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle
