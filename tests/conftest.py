import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built libmace.so")


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree; skip nothing: a GPU test without the
    library or a GPU fails loudly."""
    import torch
    from paper_1911_09278_gb300 import build as gbuild
    import paper_1911_09278_gb300 as mace
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    gbuild.build()
    mace.load()
    return mace
