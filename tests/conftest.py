import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built liblbm")
    config.addinivalue_line("markers", "slow: longer CPU runs")


@pytest.fixture(scope="session")
def d3q19():
    """The D3Q19 velocity set in the library's documented order (rest, +x, -x,
    +y, -y, +z, -z, then the 12 edge vectors), written out from the lattice
    definition, for tests that take moments."""
    import numpy as np
    e = np.array([[0, 0, 0],
                  [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                  [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
                  [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
                  [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]], dtype=np.float64)
    return e
