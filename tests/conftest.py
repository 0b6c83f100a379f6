import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


GOLDEN = os.path.join(ROOT, "tests", "golden")


@pytest.fixture(scope="session")
def libvtn():
    """Build (if needed) and load the CUDA library.  Compiling needs nvcc, not a GPU."""
    from paper_2410_18740_gb300 import build, vtn
    build.build()
    return vtn.lib()


@pytest.fixture(scope="module")
def ctx(libvtn):
    import torch
    from paper_2410_18740_gb300 import vtn
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = vtn.vtn_create(0)
    yield c
    torch.cuda.synchronize()
    vtn.vtn_destroy(c)
