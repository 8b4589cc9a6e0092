import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA device (B300, sm_103a)")
    config.addinivalue_line("markers", "slow: longer CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests run in file order; the no-allocation entry point test file is
    # named to sort last.
    pass


@pytest.fixture(scope="session")
def lib():
    """The CUDA library binding (loads the in-tree shared library)."""
    from paper_2603_22553_b300 import binding
    return binding.load()
