import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: oracle runs of more than a few seconds")


import pytest  # noqa: E402


@pytest.fixture(scope="session")
def gpu_bmg():
    """The CUDA library binding; builds libbmg.so first.  Fails loudly without it."""
    import __graft_entry__
    __graft_entry__.build()
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1511_07042_gb300 import bmg
    return bmg
