import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the built CUDA library")
    config.addinivalue_line("markers", "slow: full-size workload (still seconds to a minute)")


@pytest.fixture(scope="session")
def cuda_lib():
    """The CUDA library, built in-tree; skips nothing: a GPU test without the
    library or without a GPU fails loudly."""
    import torch

    assert torch.cuda.is_available(), "GPU test collected on a machine without a CUDA device"
    import paper_2305_17813_gb300 as mk

    return mk.load()
