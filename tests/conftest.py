import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: CPU test that takes tens of seconds")


GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read_paper_iteration_counts(fname="paper_iteration_counts.txt"):
    """Rows (medium, k/2pi, n, N_iter) of a golden file: the preconditioned GMRES(20)
    iteration counts of the paper's 3-D Tables 4-6 (paper_iteration_counts.txt) or
    2-D Tables 1-3 (paper_iteration_counts_2d.txt)."""
    rows = []
    with open(os.path.join(GOLDEN, fname)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if not line:
                continue
            med, kk, n, it = line.split()
            rows.append((med, float(kk), int(n), int(it)))
    return rows


@pytest.fixture(scope="session")
def paper_iteration_counts():
    return read_paper_iteration_counts()


@pytest.fixture(scope="session")
def paper_iteration_counts_2d():
    return read_paper_iteration_counts("paper_iteration_counts_2d.txt")
