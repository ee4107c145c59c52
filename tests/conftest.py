import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def dwf():
    """The CUDA binding; builds libdwf.so if it is missing (GPU tests only)."""
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1111_5059_gb300 import build as _build
    from paper_1111_5059_gb300 import dwf as _dwf

    if not os.path.exists(_dwf.LIB_PATH):
        _build.build()
    _dwf.lib()
    return _dwf
