import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a GB300 (sm_103a) and the built CUDA library")
    config.addinivalue_line("markers", "slow: larger CPU cases")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def hs():
    """The CUDA library's binding (built in-tree on first use); GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for tests marked gpu")
    from paper_1705_07272_gb300 import build as _build
    _build.build()
    import paper_1705_07272_gb300 as m
    m.lib()
    return m
