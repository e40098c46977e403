import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: several seconds of CPU oracle work")


@pytest.fixture(scope="session")
def small_cell_oracle():
    """Oracle results on the 512-atom two-sheet cell with 200 ions (computed once)."""
    from tests import _cases
    return _cases.small_cell_oracle()
