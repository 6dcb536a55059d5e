import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running oracle pin")


def table1():
    """(c [19,3], w [19]) read from the paper's Table 1 fixture."""
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "d3q19_table1.txt"), comments="#", dtype=np.int64)
    return rows[:, 1:4], rows[:, 4] / 36.0


@pytest.fixture(scope="session")
def d3q19():
    return table1()
