import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built libvrc")
    config.addinivalue_line("markers", "slow: larger CPU case")


@pytest.fixture(scope="session")
def vrc():
    """The CUDA library binding; a GPU test fails loudly if it cannot load."""
    from paper_1706_07476_gb300 import vrc as _vrc
    _vrc.require_device()
    return _vrc
