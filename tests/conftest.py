import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _cuda_available() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _cuda_available():
        return
    skip = pytest.mark.skip(reason="no CUDA device in this container")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build_oracle()
    return oracle


@pytest.fixture(scope="session")
def hg():
    """The CUDA library binding.  On a GPU machine a missing or broken
    extension is an error, never a skip."""
    import paper_1907_02900_gb300 as hgmod
    hgmod.load()
    return hgmod
