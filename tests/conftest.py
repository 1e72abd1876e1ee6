import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def lexlib():
    """The product library, built in-tree on first use (nvcc cross-compiles
    without a GPU)."""
    from paper_2608_03473_gb300 import _build
    import paper_2608_03473_gb300 as lg
    _build.build()
    lg.load_library()
    return lg
